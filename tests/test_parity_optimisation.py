"""Hierarchy-optimisation workload (Sec. 5.1): street-corridor views at 1280x720 with log-uniform tau.

* The batch of 8 views on a 100k-leaf corridor goes through one render and one adjoint (a9), and
  every touched node's gradient row is compared with the sum of the oracle's per-view gradients.
* At full size (2M leaves, about 4M nodes) single views are compared on 64 sampled interior nodes
  that are interpolated (t in (0.05, 0.95)) or receive an interpolated child's share.
Both use the per-element bar of tests/test_parity_backward.py (1e-3 relative plus 1e-5 of the
group's largest gradient; loss weight zero at the oracle's ambiguous pixels) over mean, scale, rot,
opacity and SH.  The oracle's gradient is pinned to central finite differences on small scenes
(tests/test_oracle_pins.py)."""
import functools

import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import synth
from tests import gpu_path
from tests.test_parity_backward import check_elementwise, gpu_grads_batch, loss_weight

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def _scene(n_leaves):
    sc = synth.corridor_scene(seed=3, n_leaves=n_leaves)
    _, views = synth.optimisation_views(seed=3)
    return sc, oracle.build_tree(sc.leaves), views


def test_adjoint_of_the_eight_view_batch():
    _, h, views = _scene(100_000)
    opts = oracle.Opts()
    dh = gpu_path.upload(h)
    ws, og = [], 0
    for k, cam in enumerate(views):
        fr = oracle.render(cam, h, opts)
        w = loss_weight(fr, 30 + k)
        ws.append(w)
        og = og + oracle.backward(cam, h, fr, w, opts)
    gg = gpu_grads_batch(dh, views, opts, ws)
    rows = np.nonzero(np.abs(og).max(axis=1) > 0)[0]
    assert len(rows) > 50_000
    assert np.all(gg[np.setdiff1d(np.arange(h.n), rows)] == 0)    # untouched nodes get nothing
    check_elementwise(gg, og, rows=rows)


@pytest.mark.parametrize("view", [0, 5])
def test_adjoint_on_sampled_interior_nodes_at_full_size(view):
    _, h, views = _scene(2_000_000)
    cam = views[view]
    opts = oracle.Opts()
    dh = gpu_path.upload(h)
    fr = oracle.render(cam, h, opts)
    w = loss_weight(fr, 10 + view)
    og = oracle.backward(cam, h, fr, w, opts)
    gg = gpu_grads_batch(dh, [cam], opts, [w])
    # 64 sampled nodes: interpolated interior cut nodes and parents of interpolated cut nodes
    t = fr.t
    sel = (t > 0.05) & (t < 0.95) & (fr.rect[:, 0] >= 0)
    ids = fr.ids[sel]
    cand = np.unique(np.concatenate([ids[h.child_count[ids] > 0], h.parent[ids]]))
    cand = cand[np.abs(og[cand]).max(axis=1) > 0]
    assert len(cand) >= 64
    pick = np.random.default_rng(view).choice(cand, 64, replace=False)
    check_elementwise(gg, og, rows=pick)
