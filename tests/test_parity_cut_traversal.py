"""The traversal cut (h3dgs_set_cut_mode 2: a level-by-level descent from the root that reads only
the records of the cut and its ancestors) against the oracle's cut rule (Sec. 4.2, Eq. t_interp):
ids and weights bit-exact, on the tiny scene at every tau (leaves only to root only), on K-ary
compacted trees, on the 2M-node street corridor and on a 4M-node tree of two streets (a scan of
several waves); the number of nodes it reads equals the size of the cut plus its ancestors, counted
here from the oracle's cut.  The scan (mode 1) selects the same and reads at least those records: it
skips only rows of 256 nodes whose nodes all have a parent below tau.  Destroying a context that ran
the traversal returns all its device memory."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import gpu_path, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()
    yield
    h3dgs.h3dgs_set_cut_mode(gpu_path.context().ctx, 0)


def _visited(h, ids):
    """|cut U ancestors of the cut|: the nodes a root-down descent must read."""
    seen = np.zeros(h.n, bool)
    seen[ids] = True
    frontier = np.unique(h.parent[ids])
    frontier = frontier[frontier >= 0]
    while len(frontier):
        new = frontier[~seen[frontier]]
        seen[new] = True
        frontier = np.unique(h.parent[new])
        frontier = frontier[frontier >= 0]
    return int(seen.sum())


def _traverse_and_compare(h, cam, scan_too=True):
    ctx = gpu_path.context()
    out = {}
    for mode in ((1, 2) if scan_too else (2,)):
        h3dgs.h3dgs_set_cut_mode(ctx.ctx, mode)
        ids, t, offs = ctx.select_cut([cam])
        st = h3dgs.h3dgs_get_stats(ctx.ctx)
        assert st["device_flags"] & 0xC == 0, st["device_flags"]
        out[mode] = (ids.cpu().numpy(), t.cpu().numpy(), offs.cpu().numpy(), st["n_cut_visited"])
    h3dgs.h3dgs_set_cut_mode(ctx.ctx, 0)
    oid, ot = oracle.select_cut(cam, h, 1)
    ids, t, offs, visited = out[2]
    np.testing.assert_array_equal(ids, oid)
    np.testing.assert_array_equal(t.view(np.uint32), ot.view(np.uint32))
    assert offs[0] == 0 and offs[1] == len(oid)
    assert visited == _visited(h, oid)
    scan_read = None
    if scan_too:
        scan_read = out[1][3]
        assert visited <= scan_read <= h.n
        np.testing.assert_array_equal(out[1][0], ids)
        np.testing.assert_array_equal(out[1][1].view(np.uint32), t.view(np.uint32))
    return oid, visited, scan_read


@pytest.mark.parametrize("tau", [0.0, 2.0, 6.0, 15.0, 80.0, float("inf")])
def test_tiny_scene(tau):
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    oid, visited, _ = _traverse_and_compare(h, synth.with_tau(sc.cameras[0], tau))
    if tau == float("inf"):
        assert list(oid) == [0] and visited == 1


def test_camera_inside_the_root_box_and_off_axis_views():
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    for cam in (synth.look_camera([5.0, 5.0, 5.0], [0.3, 0.2, 1.0], [0, -1, 0], 160, 120, 70.0, 4.0),
                synth.look_camera([-8, 5, 5.0], [1, 0, 0.05], [0, -1, 0], 96, 128, 75.0, 15.0)):
        _traverse_and_compare(h, cam)


@pytest.mark.parametrize("tau", [3.0, 15.0])
def test_compacted_k_ary_tree(tau):
    from tests.test_parity_compaction import _tiny_views
    sc, h = scenes.tiny()
    oh, _ = oracle.compact(_tiny_views(), h, 3.0, 128.0)
    assert oh.child_count.max() > 2
    gpu_path.upload(oh)
    _traverse_and_compare(oh, synth.with_tau(sc.cameras[0], tau))


@pytest.mark.slow
@pytest.mark.parametrize("tau", [0.0, 3.0, 6.0, 15.0])
def test_street_corridor_full_size(tau):
    sc, h = scenes.corridor()
    gpu_path.upload(h)
    oid, visited, _ = _traverse_and_compare(h, synth.with_tau(sc.cameras[0], tau))
    assert visited == 2 * len(oid) - 1   # binary tree: the cut's ancestors are one fewer than the cut


@pytest.mark.slow
@pytest.mark.parametrize("tau,max_read", [(3.0, 1.0), (6.0, 0.4), (15.0, 0.1)])
def test_scan_skips_rows_below_the_cut(tau, max_read):
    """From high above the street most rows of the deep levels have every parent below tau: the scan
    skips them unread (a bound of their parents' granularity from the union box and the largest side)
    and still selects the oracle's cut and weights bit for bit.  (A row holding any child of an
    expanded node is read; at tau = 3 nearly every row holds one.)"""
    sc, h = scenes.corridor()
    gpu_path.upload(h)
    lo, hi = h.box_min[0].astype(np.float64), h.box_max[0].astype(np.float64)
    centre = 0.5 * (lo + hi)
    pos = centre + np.array([0.0, 0.0, 0.6 * float(np.max(hi - lo))])
    cam = synth.look_camera(pos, [0.05, 0.0, -1.0], [1.0, 0.0, 0.0], 1920, 1080, 60.0, tau)
    oid, visited, scan_read = _traverse_and_compare(h, cam)
    assert len(oid) > 1000
    assert scan_read <= max_read * h.n



@pytest.mark.slow
@pytest.mark.parametrize("tau", [3.0, 6.0, 15.0])
def test_scan_of_several_waves(tau):
    """A tree of more than six scan tiles per SM (the scan's longer tiles, several waves of blocks
    chained by the look-back, the row skipping): the default mode, the forced scan and the traversal
    all select the oracle's nodes and weights bit for bit, over both copies of the street."""
    sc, _ = scenes.corridor()
    h = scenes.two_corridors()
    assert h.n == 2 * scenes.corridor()[1].n + 1
    gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], tau)
    ctx = gpu_path.context()
    ids0, t0, offs0 = ctx.select_cut([cam])
    assert h3dgs.h3dgs_get_stats(ctx.ctx)["device_flags"] & 0xC == 0
    oid, visited, scan_read = _traverse_and_compare(h, cam)
    np.testing.assert_array_equal(ids0.cpu().numpy(), oid)
    np.testing.assert_array_equal(t0.cpu().numpy().view(np.uint32), oracle.select_cut(cam, h, 1)[1].view(np.uint32))
    assert int(offs0[1]) == len(oid) > 1000
    # both copies contribute (the second one, shifted down the street, is seen far away)
    n1 = scenes.corridor()[1].n
    assert np.any(oid >= n1 + 2) and np.any((oid >= 3) & (oid < n1 + 2))

@pytest.mark.slow
def test_destroy_returns_every_device_buffer():
    """A context that ran the traversal cut and a render gives all its device memory back when it is
    destroyed: the free memory the driver reports returns to its level before the context (the same
    work ran once before, so that loading the kernels' code is not counted)."""
    import torch
    sc, h = scenes.corridor()
    dh = h3dgs.DeviceHierarchy.from_arrays(h)
    cam = sc.cameras[0]

    def run_once():
        ctx = h3dgs.Context(torch.cuda.current_device())
        ctx.upload(dh)
        h3dgs.h3dgs_set_cut_mode(ctx.ctx, 2)
        cut = ctx.select_cut([cam])
        img = ctx.render([cam], cut)
        torch.cuda.synchronize()
        assert h3dgs.h3dgs_get_stats(ctx.ctx)["device_flags"] == 0
        del cut, img
        ctx.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    run_once()
    free0 = torch.cuda.mem_get_info()[0]
    run_once()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 8 << 20, (free0 - free1) / 2**20
