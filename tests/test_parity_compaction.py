"""Parity of the device compaction (h3dgs_compact_hierarchy, Sec. 5.2) with the oracle, and of the
render path and its adjoint on compacted trees, whose nodes have K > 2 children (the transition
opacity 1 - (1 - alpha_p)^(1/K)).

Bars: node order, topology and the old index of every node bit-exact; attribute rows and boxes
bit-exact (they are copied); renders and gradients on the compacted tree at the forward and
backward parity bars."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import gpu_path, scenes
from tests.test_parity_backward import _check, _gpu_grads, loss_weight
from tests.test_parity_forward import _compare

pytestmark = pytest.mark.gpu
FIELDS = ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start", "child_count")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _device_vs_oracle(h, cams, tau_min, tau_max):
    gpu_path.upload(h)
    dh, old = gpu_path.context().compact(cams, tau_min, tau_max)
    oh, oold = oracle.compact(cams, h, tau_min, tau_max)
    np.testing.assert_array_equal(old.cpu().numpy(), oold)
    for k in FIELDS:
        g = getattr(dh, k).cpu().numpy()
        o = getattr(oh, k)
        np.testing.assert_array_equal(g.view(np.uint32) if g.dtype == np.float32 else g,
                                      o.view(np.uint32) if o.dtype == np.float32 else o, err_msg=k)
    return oh, oold


def _tiny_views():
    return synth.orbit_views([5.0, 5.0, 5.0], 14.0, 12, 256, 256, seed=2)


@pytest.mark.parametrize("tau_min,tau_max,removes", [(3.0, 128.0, True), (1.0, 512.0, True), (0.25, 2.0, False),
                                                   (8.0, 4.0, False)])
def test_tiny_tree(tau_min, tau_max, removes):
    sc, h = scenes.tiny()
    oh, old = _device_vs_oracle(h, _tiny_views(), tau_min, tau_max)
    assert (oh.n < h.n) == removes


def test_flattened_tree_and_single_view():
    sc, h = scenes.tiny()
    far = synth.look_camera([5.0, 5.0, -2.0e4], [0, 0, 1], [0, -1, 0], 256, 256, 60.0, 6.0)
    oh, old = _device_vs_oracle(h, [far], 3.0, 128.0)
    assert oh.n == 1 + int(np.sum(h.child_count == 0))
    _device_vs_oracle(h, sc.cameras, 3.0, 128.0)


def test_many_views_over_several_shared_memory_rounds():
    sc, h = scenes.tiny()
    cams = synth.orbit_views([5.0, 5.0, 5.0], 30.0, 1100, 64, 64, seed=4)
    _device_vs_oracle(h, cams, 2.0, 64.0)


def test_corridor_full_size():
    """The 1M-leaf corridor (2M nodes) with 32 training views along the street, tau in [3, 960]."""
    sc, h = scenes.corridor()
    cams = synth.corridor_views(n_views=32)
    oh, old = _device_vs_oracle(h, cams, 3.0, 960.0)
    assert oh.n < h.n and oh.child_count.max() > 2


def test_capacity_and_argument_errors():
    import torch
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    ctx = gpu_path.context()
    cams = _tiny_views()
    oh, _ = oracle.compact(cams, h, 3.0, 128.0)
    f = lambda *s: torch.empty(s, dtype=torch.float32, device="cuda")
    i = lambda n: torch.empty(n, dtype=torch.int32, device="cuda")
    small = oh.n - 1
    out = h3dgs.DeviceHierarchy(f(small, 3), f(small, 3), f(small, 4), f(small), f(small, 48), f(small, 3),
                                f(small, 3), i(small), i(small), i(small))
    with pytest.raises(h3dgs.H3dgsError) as e:
        h3dgs.h3dgs_compact_hierarchy(ctx.ctx, cams, 3.0, 128.0, out)
    assert e.value.status == 4
    for bad in ((0.0, 128.0), (3.0, float("inf")), (1e-30, 1e30)):
        with pytest.raises(h3dgs.H3dgsError) as e:
            h3dgs.h3dgs_compact_hierarchy(ctx.ctx, cams, *bad, out)
        assert e.value.status == 1
    with pytest.raises(h3dgs.H3dgsError) as e:   # output overlapping the resident hierarchy
        h3dgs.h3dgs_compact_hierarchy(ctx.ctx, cams, 3.0, 128.0, ctx.hier)
    assert e.value.status == 1
    # the context still renders after the refused calls
    _device_vs_oracle(h, cams, 3.0, 128.0)


@pytest.fixture(scope="module")
def compacted_tiny():
    sc, h = scenes.tiny()
    oh, _ = oracle.compact(_tiny_views(), h, 3.0, 128.0)
    return sc, oh


@pytest.mark.parametrize("tau", [3.0, 6.0, 15.0, 40.0])
def test_render_on_compacted_tree(compacted_tiny, tau):
    sc, oh = compacted_tiny
    cam = synth.with_tau(sc.cameras[0], tau)
    dh = gpu_path.upload(oh)
    ofr, g = _compare(cam, oh, dh, oracle.Opts())
    if tau in (6.0, 15.0):
        wide = oh.child_count[np.maximum(oh.parent[ofr.ids], 0)] > 2
        assert np.sum(wide & (ofr.t > 0.05) & (ofr.t < 0.95)) > 0


@pytest.mark.parametrize("tau", [6.0, 15.0])
def test_backward_on_compacted_tree(compacted_tiny, tau):
    sc, oh = compacted_tiny
    cam = synth.with_tau(sc.cameras[0], tau)
    opts = oracle.Opts()
    dh = gpu_path.upload(oh)
    fr = oracle.render(cam, oh, opts)
    w = loss_weight(fr, 3)
    og = oracle.backward(cam, oh, fr, w, opts)
    gg = _gpu_grads(dh, cam, opts, w)
    _check(gg, og)
