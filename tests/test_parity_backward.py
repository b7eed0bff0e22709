"""Parity of the CUDA adjoint (h3dgs_render_backward) with the oracle's fp64 analytic gradient.

Bar: for each attribute group (mean, scale, rot, opacity, sh) the largest absolute difference is
at most 1e-3 of the group's largest oracle gradient, and the relative L2 error of the group is at
most 1e-3.  The oracle's gradient is itself pinned to central finite differences
(tests/test_oracle_pins.py).
"""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import gpu_path, scenes

pytestmark = pytest.mark.gpu

GROUPS = [("mean", 0, 3), ("scale", 3, 6), ("rot", 6, 10), ("opacity", 10, 11), ("sh", 11, 59)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _gpu_grads(dh, cam, opts, w, freeze=0, chunk=None):
    import torch
    fr = gpu_path.run(dh, [cam], opts, debug=False, chunk=chunk)  # keeps the cut buffers alive (re-read by the backward)
    grads = {k: torch.zeros_like(getattr(dh, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dl = torch.from_numpy(np.ascontiguousarray(w, np.float32).reshape(-1)).cuda()
    h3dgs.h3dgs_render_backward(gpu_path.context().ctx, dl, grads, freeze)
    torch.cuda.synchronize()
    del fr
    return np.concatenate([grads[k].cpu().numpy().reshape(dh.n, -1) for k in ("mean", "scale", "rot", "opacity", "sh")],
                          axis=1)


def _check(gg, og, tol=1e-3):
    for name, a, b in GROUPS:
        o, g = og[:, a:b], gg[:, a:b]
        scale = np.abs(o).max()
        if scale == 0:
            assert np.abs(g).max() == 0, name
            continue
        assert np.abs(g - o).max() <= tol * scale, (name, np.abs(g - o).max() / scale)
        assert np.linalg.norm(g - o) <= tol * np.linalg.norm(o), (name, np.linalg.norm(g - o) / np.linalg.norm(o))


def _fd_scene():
    lv, cam = scenes.small_random_scene(n_leaves=40, res=(40, 32), seed=9, log_scale=-2.2)
    h = oracle.build_tree(lv)
    eps = oracle.granularity(cam, h)
    tau = float(np.quantile(eps[h.child_count > 0], 0.5))
    return h, synth.with_tau(cam, tau)


@pytest.mark.parametrize("freeze", [0, 1])
def test_backward_small_interpolated_scene(freeze):
    h, cam = _fd_scene()
    opts = oracle.Opts()
    dh = gpu_path.upload(h)
    fr = oracle.render(cam, h, opts)
    assert np.sum((fr.t > 0.05) & (fr.t < 0.95)) >= 3
    w = np.random.default_rng(0).normal(size=fr.image.shape)
    og = oracle.backward(cam, h, fr, w, opts, freeze_leaves=freeze)
    gg = _gpu_grads(dh, cam, opts, w, freeze)
    _check(gg, og)
    if freeze:
        assert np.all(gg[h.child_count == 0] == 0)


@pytest.mark.parametrize("tau,chunk", [(0.0, None), (6.0, None), (30.0, None), (2.0, 64), (6.0, 100)])
def test_backward_tiny_scene(tau, chunk):
    sc, h = scenes.tiny()
    cam = synth.with_tau(sc.cameras[0], tau)
    opts = oracle.Opts()
    dh = gpu_path.upload(h)
    fr = oracle.render(cam, h, opts)
    w = np.random.default_rng(1).normal(size=fr.image.shape)
    og = oracle.backward(cam, h, fr, w, opts)
    gg = _gpu_grads(dh, cam, opts, w, chunk=chunk)
    _check(gg, og)


def test_backward_options():
    sc, h = scenes.tiny()
    cam = synth.with_tau(sc.cameras[0], 6.0)
    dh = gpu_path.upload(h)
    for opts in (oracle.Opts(interpolate=0), oracle.Opts(aa_compensate=0, bg=(0.3, 0.1, 0.9)),
                 oracle.Opts(tile_w=8, tile_h=8)):
        fr = oracle.render(cam, h, opts)
        w = np.random.default_rng(2).normal(size=fr.image.shape)
        og = oracle.backward(cam, h, fr, w, opts)
        gg = _gpu_grads(dh, cam, opts, w)
        _check(gg, og)
