"""Streamed hierarchy (h3dgs_upload_hierarchy_streamed, h3dgs_stream_update / _cleanup; Sec. 6.3)
against the oracle's residency trace and against the resident render.

Bars: the number of nodes transferred by every update and the resident count after every cleanup
equal the oracle's trace exactly; every streamed frame is bit-identical to the resident render of
the same cut (the cache holds the same floats)."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _walk(h, cams, cache, update_every, cleanup_every, max_age):
    import torch
    res = h3dgs.Context(torch.cuda.current_device())
    stm = h3dgs.Context(torch.cuda.current_device())
    try:
        dh = h3dgs.DeviceHierarchy.from_arrays(h)
        res.upload(dh)
        stm.upload_streamed(dh, cache)
        transfers, after = [], []
        cut = None
        for f, cam in enumerate(cams):
            if f % update_every == 0:
                cut = stm.select_cut([cam])
                transfers.append(h3dgs.h3dgs_stream_update(stm.ctx, 1, *cut, f))
            a = stm.render([cam], cut)
            b = res.render([cam], cut)
            torch.cuda.synchronize()
            assert h3dgs.h3dgs_get_stats(stm.ctx)["device_flags"] == 0
            assert torch.equal(a, b), f"frame {f} differs from the resident render"
            if (f + 1) % cleanup_every == 0:
                after.append(h3dgs.h3dgs_stream_cleanup(stm.ctx, f, max_age))
        return transfers, after
    finally:
        stm.close()
        res.close()


@pytest.mark.parametrize("update_every,cleanup_every,max_age", [(2, 100, 100), (2, 4, 2), (1, 3, 0)])
def test_tiny_orbit(update_every, cleanup_every, max_age):
    sc, h = scenes.tiny()
    cams = synth.orbit_views([5.0, 5.0, 5.0], 14.0, 12, 200, 150, tau=4.0, seed=5)
    tr, after = _walk(h, cams, h.n, update_every, cleanup_every, max_age)
    otr, oafter, _ = oracle.stream_trace(cams, h, update_every, cleanup_every, max_age)
    assert tr == otr
    assert after == oafter


def test_corridor_drive():
    """The 1M-leaf corridor (2M nodes), 16 poses 3 m apart along the street, cut every 2 frames,
    cleanup every 8 frames."""
    sc, h = scenes.corridor()
    line = synth.corridor_polyline(1)
    cams = [synth.corridor_camera(line, 300.0 + 3.0 * i, 960, 540, 6.0) for i in range(16)]
    tr, after = _walk(h, cams, h.n // 2, 2, 8, 4)
    otr, oafter, _ = oracle.stream_trace(cams, h, 2, 8, 4)
    assert tr == otr and after == oafter
    assert tr[0] > 10 * max(tr[1:])   # a short step needs few new nodes


def test_cache_too_small_is_reported_and_the_frame_flags_absent_nodes():
    import torch
    sc, h = scenes.tiny()
    cam = sc.cameras[0]
    stm = h3dgs.Context(torch.cuda.current_device())
    try:
        stm.upload_streamed(h3dgs.DeviceHierarchy.from_arrays(h), 64)
        cut = stm.select_cut([cam])
        with pytest.raises(h3dgs.H3dgsError) as e:
            h3dgs.h3dgs_stream_update(stm.ctx, 1, *cut, 0)
        assert e.value.status == 4
        stm.render([cam], cut)
        torch.cuda.synchronize()
        assert h3dgs.h3dgs_get_stats(stm.ctx)["device_flags"] & 0x20
        # the adjoint refuses a streamed hierarchy
        stm.render([cam], cut, save_for_backward=1)
        g = {k: torch.zeros(1, device="cuda") for k in ("mean", "scale", "rot", "opacity", "sh")}
        with pytest.raises(h3dgs.H3dgsError) as e:
            h3dgs.h3dgs_render_backward(stm.ctx, torch.zeros(3 * cam.width * cam.height, device="cuda"), g, 0)
        assert e.value.status == 6
        # a full cleanup frees every row
        assert h3dgs.h3dgs_stream_cleanup(stm.ctx, 10, 0) == 0
    finally:
        stm.close()
