"""Parity of the CUDA adjoint (h3dgs_render_backward) with the oracle's fp64 analytic gradient.

Bar, per element of every attribute group (mean, scale, rot, opacity, sh):
    |g - o| <= 1e-3 |o| + FLOOR * max|o over the group|,
and the relative L2 error of each group at most 1e-3.  FLOOR (1e-5) is the absolute allowance for
elements that are sums of many terms of both signs, where fp32 accumulation in a different order
leaves an error proportional to the terms rather than to their sum.  The loss weight is zero at the
pixels whose fp32 decisions the oracle flags as ambiguous (within 1e-5 of the alpha floor or the
transmittance stop), the pixels the image bar excludes too.  The oracle's gradient is itself pinned
to central finite differences (tests/test_oracle_pins.py).
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
    return gpu_grads_batch(dh, [cam], opts, [w], freeze, chunk)


def gpu_grads_batch(dh, cams, opts, ws, freeze=0, chunk=None):
    """One h3dgs_render(save_for_backward = 1) of all cameras, then one h3dgs_render_backward with
    the packed per-camera image gradients ws; returns the node gradient rows [N, 59]."""
    import torch
    fr = gpu_path.run(dh, cams, opts, debug=False, chunk=chunk)  # keeps the cut buffers alive (re-read by the backward)
    grads = {k: torch.zeros_like(getattr(dh, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dl = torch.from_numpy(np.concatenate([np.ascontiguousarray(w, np.float32).reshape(-1) for w in ws])).cuda()
    h3dgs.h3dgs_render_backward(gpu_path.context().ctx, dl, grads, freeze)
    torch.cuda.synchronize()
    flags = h3dgs.h3dgs_get_stats(gpu_path.context().ctx)["device_flags"]
    assert flags & 0x88 == 0, (flags, h3dgs.h3dgs_last_error(gpu_path.context().ctx))
    del fr
    return np.concatenate([grads[k].cpu().numpy().reshape(dh.n, -1) for k in ("mean", "scale", "rot", "opacity", "sh")],
                          axis=1)


FLOOR = 1e-5


def check_elementwise(gg, og, rtol=1e-3, floor=FLOOR, rows=None):
    """Per-element bar above; returns the worst (|g - o| - rtol |o|) / max|o| per group."""
    worst = {}
    for name, a, b in GROUPS:
        o = og[:, a:b] if rows is None else og[rows, a:b]
        g = gg[:, a:b] if rows is None else gg[rows, a:b]
        scale = np.abs(o).max()
        if scale == 0:
            assert np.abs(g).max() == 0, name
            continue
        excess = (np.abs(g - o) - rtol * np.abs(o)) / scale
        worst[name] = float(excess.max())
        assert excess.max() <= floor, (name, float(excess.max()), np.unravel_index(np.argmax(excess), excess.shape))
        assert np.linalg.norm(g - o) <= rtol * np.linalg.norm(o), (name, np.linalg.norm(g - o) / np.linalg.norm(o))
    return worst


_check = check_elementwise


def loss_weight(fr, seed):
    """A seeded dL/dimage, zero at the oracle's ambiguous pixels."""
    w = np.random.default_rng(seed).normal(size=fr.image.shape)
    w[:, fr.ambiguous] = 0.0
    return w


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
    w = loss_weight(fr, 0)
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
    w = loss_weight(fr, 1)
    og = oracle.backward(cam, h, fr, w, opts)
    gg = _gpu_grads(dh, cam, opts, w, chunk=chunk)
    _check(gg, og)



@pytest.mark.parametrize("seed", range(10))
def test_backward_random_scenes_and_cameras(seed):
    """The adjoint on the forward path's seeded random scenes and cameras (inside or outside the
    scene, ragged resolutions, one frame that sees nothing)."""
    h, cam = scenes.random_case(seed)
    opts = oracle.Opts()
    dh = gpu_path.upload(h)
    fr = oracle.render(cam, h, opts)
    w = loss_weight(fr, 10 + seed)
    og = oracle.backward(cam, h, fr, w, opts)
    gg = _gpu_grads(dh, cam, opts, w)
    _check(gg, og)

def test_backward_options():
    sc, h = scenes.tiny()
    cam = synth.with_tau(sc.cameras[0], 6.0)
    dh = gpu_path.upload(h)
    for opts in (oracle.Opts(interpolate=0), oracle.Opts(aa_compensate=0, bg=(0.3, 0.1, 0.9)),
                 oracle.Opts(tile_w=8, tile_h=8)):
        fr = oracle.render(cam, h, opts)
        w = loss_weight(fr, 2)
        og = oracle.backward(cam, h, fr, w, opts)
        gg = _gpu_grads(dh, cam, opts, w)
        _check(gg, og)


def test_backward_multi_camera_equals_sum_of_views():
    """Three cameras of different resolution and tau in one render + one adjoint (a9): every node's
    gradient is the sum of its gradients in the three views (shared interior nodes collect from
    several views, as in the hierarchy optimisation of Sec. 5.1)."""
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    opts = oracle.Opts()
    cams = [synth.with_tau(sc.cameras[0], 6.0),
            synth.look_camera([5, 5, -12.0], [0.1, 0, 1], [0, -1, 0], 200, 150, 60.0, 3.0),
            synth.look_camera([-8, 5, 5.0], [1, 0, 0.05], [0, -1, 0], 96, 128, 75.0, 15.0)]
    ws, og = [], 0
    for k, cam in enumerate(cams):
        fr = oracle.render(cam, h, opts)
        w = loss_weight(fr, 20 + k)
        ws.append(w)
        og = og + oracle.backward(cam, h, fr, w, opts)
    gg = gpu_grads_batch(dh, cams, opts, ws)
    _check(gg, og)
    # nodes that two or more views reach exist and are covered by the bar above
    reach = [np.abs(oracle.backward(c, h, oracle.render(c, h, opts), np.ones((3, c.height, c.width)), opts)).max(1) > 0
             for c in cams]
    assert np.sum(np.sum(reach, axis=0) >= 2) > 100
