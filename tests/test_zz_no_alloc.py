"""The allocation-free cut entry point agrees with the context entry point.

h3dgs_select_cut_noalloc serves callers that cannot allocate device memory (another framework owns
the memory budget, or the loop must not enter the driver's allocator); its scratch is a fixed
array inside the library.  This file is collected last so that a failure here cannot hide any other
test in a run that stops at the first failure.  It passes alone in a fresh process too.
"""
import numpy as np
import pytest

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


def _both(dh, cam):
    import torch
    ctx = gpu_path.context()
    ids, t, offs = ctx.select_cut([cam])
    cap = dh.n
    ids2 = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    t2 = torch.full((cap,), -7.0, dtype=torch.float32, device="cuda")
    offs2 = torch.full((2,), -7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    total = h3dgs.h3dgs_select_cut_noalloc(dh, cam, ids2, t2, offs2, cap, stream)
    torch.cuda.synchronize()
    return (ids.cpu().numpy(), t.cpu().numpy(), offs.cpu().numpy()), \
           (ids2[:total].cpu().numpy(), t2[:total].cpu().numpy(), offs2.cpu().numpy(), total)


def test_noalloc_cut_matches_context_cut_on_consecutive_calls():
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    # two calls in a row with different results: the shared scratch keeps the previous call's
    # contents, which must not leak into the next
    for cam in (synth.with_tau(sc.cameras[0], 6.0), synth.with_tau(sc.cameras[0], 1.5),
                synth.look_camera([5.0, 5.0, 5.0], [0.3, 0.2, 1.0], [0, -1, 0], 160, 120, 70.0, 4.0)):
        (ids, t, offs), (ids2, t2, offs2, total) = _both(dh, cam)
        assert total == len(ids) == offs2[1] and offs2[0] == 0
        np.testing.assert_array_equal(ids2, ids)
        np.testing.assert_array_equal(t2.view(np.uint32), t.view(np.uint32))



@pytest.mark.parametrize("seed", range(10))
def test_noalloc_cut_on_random_scenes_and_cameras(seed):
    """On the forward path's seeded random scenes and cameras the allocation-free cut equals the
    oracle's cut rule, ids and weights bit for bit."""
    import oracle
    h, cam = scenes.random_case(seed)
    dh = gpu_path.upload(h)
    _, (ids2, t2, offs2, total) = _both(dh, cam)
    oid, ot = oracle.select_cut(cam, h, 1)
    assert total == len(oid) == offs2[1]
    np.testing.assert_array_equal(ids2, oid)
    np.testing.assert_array_equal(t2.view(np.uint32), ot.view(np.uint32))

def test_noalloc_cut_on_the_two_million_node_corridor():
    sc, h = scenes.corridor()
    dh = gpu_path.upload(h)
    for tau in (6.0, 15.0):
        (ids, t, _), (ids2, t2, offs2, total) = _both(dh, synth.with_tau(sc.cameras[0], tau))
        np.testing.assert_array_equal(ids2, ids)
        np.testing.assert_array_equal(t2.view(np.uint32), t.view(np.uint32))


def test_noalloc_rejects_trees_beyond_its_scratch():
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    ids = torch.empty(8, dtype=torch.int32, device="cuda")
    offs = torch.empty(2, dtype=torch.int64, device="cuda")
    with pytest.raises(h3dgs.H3dgsError) as e:
        h3dgs.h3dgs_select_cut_noalloc(dh, sc.cameras[0], ids, None, offs, 8,
                                       n_nodes=(1 << 24) + 1)
    assert e.value.status == 4   # H3DGS_ERR_CAPACITY, nothing launched


def test_noalloc_truncates_at_capacity_and_reports_the_full_size():
    """A capacity below the cut size: the first `capacity` ids are written, the end offset is clamped
    to the capacity, and the call returns H3DGS_ERR_CAPACITY after storing the untruncated size."""
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], 1.5)
    ids, _, _ = gpu_path.context().select_cut([cam])
    ids = ids.cpu().numpy()
    cap = len(ids) // 3
    assert cap > 32
    ids2 = torch.full((cap + 16,), -7, dtype=torch.int32, device="cuda")
    offs2 = torch.full((2,), -7, dtype=torch.int64, device="cuda")
    with pytest.raises(h3dgs.H3dgsError) as e:
        h3dgs.h3dgs_select_cut_noalloc(dh, cam, ids2, None, offs2, cap, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert e.value.status == 4           # H3DGS_ERR_CAPACITY
    assert e.value.total == len(ids)
    o = offs2.cpu().numpy()
    assert o[0] == 0 and o[1] == cap
    got = ids2.cpu().numpy()
    np.testing.assert_array_equal(got[:cap], ids[:cap])
    assert np.all(got[cap:] == -7)        # nothing written beyond the capacity


def test_noalloc_without_total_does_not_synchronise_and_matches_after_a_sync():
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], 4.0)
    ids, t, offs = gpu_path.context().select_cut([cam])
    cap = dh.n
    ids2 = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    t2 = torch.full((cap,), -7.0, dtype=torch.float32, device="cuda")
    offs2 = torch.full((2,), -7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    assert h3dgs.h3dgs_select_cut_noalloc(dh, cam, ids2, t2, offs2, cap, stream.cuda_stream,
                                          want_total=False) is None
    stream.synchronize()
    n = int(offs2[1].item())
    assert n == len(ids) and int(offs2[0].item()) == 0
    np.testing.assert_array_equal(ids2[:n].cpu().numpy(), ids.cpu().numpy())
    np.testing.assert_array_equal(t2[:n].cpu().numpy().view(np.uint32), t.cpu().numpy().view(np.uint32))
