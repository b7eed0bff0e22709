"""Hierarchy-optimisation workload at full size: 2M-leaf street corridor (about 4M nodes), 1280x720
views at log-uniform tau (Sec. 5.1).  The oracle builds the hierarchy; the adjoint is compared with the
oracle's fp64 analytic gradient on 64 sampled interior nodes that are interpolated (t in (0.05, 0.95))
or receive an interpolated child's share, over mean, scale, rot, opacity and SH.  The oracle's
gradient is pinned to central finite differences on small scenes (tests/test_oracle_pins.py)."""
import functools

import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import gpu_path

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
GROUPS = [("mean", 0, 3), ("scale", 3, 6), ("rot", 6, 10), ("opacity", 10, 11), ("sh", 11, 59)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def _scene():
    sc = synth.corridor_scene(seed=3, n_leaves=2_000_000)
    _, views = synth.optimisation_views(seed=3)
    return sc, oracle.build_tree(sc.leaves), views


@pytest.mark.parametrize("view", [0, 5])
def test_adjoint_on_sampled_interior_nodes_at_full_size(view):
    import torch
    sc, h, views = _scene()
    cam = views[view]
    opts = oracle.Opts()
    dh = gpu_path.upload(h)
    fr = oracle.render(cam, h, opts)
    w = np.random.default_rng(10 + view).normal(size=fr.image.shape)
    og = oracle.backward(cam, h, fr, w, opts)
    g = gpu_path.run(dh, [cam], opts, debug=False)   # keeps the cut buffers alive for the adjoint
    grads = {k: torch.zeros_like(getattr(dh, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dl = torch.from_numpy(np.ascontiguousarray(w, np.float32).reshape(-1)).cuda()
    h3dgs.h3dgs_render_backward(gpu_path.context().ctx, dl, grads, 0)
    torch.cuda.synchronize()
    gg = np.concatenate([grads[k].cpu().numpy().reshape(dh.n, -1) for k in ("mean", "scale", "rot", "opacity", "sh")],
                        axis=1)
    del g
    # 64 sampled nodes: interpolated interior cut nodes and parents of interpolated cut nodes
    t = fr.t
    sel = (t > 0.05) & (t < 0.95) & (fr.rect[:, 0] >= 0)
    ids = fr.ids[sel]
    cand = np.unique(np.concatenate([ids[h.child_count[ids] > 0], h.parent[ids]]))
    cand = cand[np.abs(og[cand]).max(axis=1) > 0]
    assert len(cand) >= 64
    pick = np.random.default_rng(view).choice(cand, 64, replace=False)
    for name, a, b in GROUPS:
        o, gq = og[pick, a:b], gg[pick, a:b]
        scale = np.abs(o).max()
        assert scale > 0, name
        assert np.abs(gq - o).max() <= 1e-3 * scale, (name, np.abs(gq - o).max() / scale)
        assert np.linalg.norm(gq - o) <= 1e-3 * np.linalg.norm(o), (name, np.linalg.norm(gq - o) / np.linalg.norm(o))
