"""Failure paths of the library, made on the host or through bounded device waits (nothing faults,
traps or hangs the GPU): argument checks, state errors, capacity overflow reported through the
device flags, non-finite attributes, and a device wait that gives up and leaves the context usable."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import gpu_path, scenes

pytestmark = pytest.mark.gpu
INVALID_ARG, CAPACITY, STATE = 1, 4, 6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _status(fn, *a, **k):
    with pytest.raises(h3dgs.H3dgsError) as e:
        fn(*a, **k)
    return e.value.status


def test_invalid_arguments_are_rejected_before_any_launch():
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    ctx = gpu_path.context()
    cam = sc.cameras[0]
    cut = ctx.select_cut([cam])
    img = torch.empty(3 * cam.width * cam.height, device="cuda")
    ids, t, offs = cut
    for bad in (dict(tile_w=16, tile_h=4), dict(tile_w=12, tile_h=16), dict(blend_chunk=10),
                dict(alpha_clamp=1.5), dict(lowpass=-1.0)):
        assert _status(h3dgs.h3dgs_render, ctx.ctx, [cam], ids, t, offs, h3dgs.default_opts(**bad), img) == INVALID_ARG
    bad_cam = synth.Camera(cam.R, cam.T, 0.0, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.tau)
    assert _status(h3dgs.h3dgs_select_cut, ctx.ctx, [bad_cam], ids, t, offs, len(ids)) == INVALID_ARG
    empty_cam = synth.Camera(cam.R, cam.T, cam.fx, cam.fy, cam.cx, cam.cy, 0, cam.height, cam.tau)
    assert _status(h3dgs.h3dgs_select_cut, ctx.ctx, [empty_cam], ids, t, offs, len(ids)) == INVALID_ARG
    assert _status(h3dgs.h3dgs_debug_wait_timeout, ctx.ctx, 0) == INVALID_ARG
    # misaligned gradient rows for the vector reductions
    ctx.render([cam], cut, save_for_backward=1)
    grads = {k: torch.zeros_like(getattr(dh, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    grads["sh"] = torch.zeros(dh.sh.numel() + 1, device="cuda")[1:].view_as(dh.sh)
    assert _status(h3dgs.h3dgs_render_backward, ctx.ctx, torch.zeros_like(img), grads, 0) == INVALID_ARG


def test_backward_without_a_saved_forward_is_a_state_error():
    import torch
    sc, h = scenes.tiny()
    ctx = h3dgs.Context(torch.cuda.current_device())
    try:
        dh = h3dgs.DeviceHierarchy.from_arrays(h)
        ctx.upload(dh)
        grads = {k: torch.zeros_like(getattr(dh, k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
        dl = torch.zeros(3 * 256 * 256, device="cuda")
        assert _status(h3dgs.h3dgs_render_backward, ctx.ctx, dl, grads, 0) == STATE
        ctx.render(sc.cameras, ctx.select_cut(sc.cameras), save_for_backward=0)
        assert _status(h3dgs.h3dgs_render_backward, ctx.ctx, dl, grads, 0) == STATE
    finally:
        ctx.close()


def test_capacity_overflow_is_reported_not_faulted():
    import torch
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    ctx = gpu_path.context()
    cam = sc.cameras[0]
    full = ctx.select_cut([cam])
    m = len(full[0])
    ids = torch.empty(m // 2, dtype=torch.int32, device="cuda")
    t = torch.empty(m // 2, dtype=torch.float32, device="cuda")
    offs = torch.empty(2, dtype=torch.int64, device="cuda")
    assert _status(h3dgs.h3dgs_select_cut, ctx.ctx, [cam], ids, t, offs, m // 2) == CAPACITY
    # a fixed workspace too small for the pairs: the frame is flagged, the next unreserved frame is fine
    img = torch.empty(3 * cam.width * cam.height, device="cuda")
    try:
        h3dgs.h3dgs_reserve(ctx.ctx, m + 16, 64)
        ctx.render([cam], full, images=img)
        torch.cuda.synchronize()
        assert h3dgs.h3dgs_get_stats(ctx.ctx)["device_flags"] & 0x1
    finally:
        h3dgs.h3dgs_reserve(ctx.ctx, 0, 0)
    full = ctx.select_cut([cam])   # a new cut clears the truncation flag of the short one above
    ctx.render([cam], full, images=img)
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    assert st["device_flags"] == 0
    fr = oracle.render(cam, h, oracle.Opts())
    im = img.view(3, cam.height, cam.width).cpu().numpy()
    assert np.abs(im - fr.image).max(axis=0)[~fr.ambiguous].max() <= 2e-3


def test_non_finite_attributes_are_culled_or_skipped():
    import torch
    sc, h = scenes.tiny()
    dh = h3dgs.DeviceHierarchy.from_arrays(h)
    rng = np.random.default_rng(5)
    for k in ("mean", "scale", "rot", "opacity", "sh"):
        a = getattr(dh, k)
        rows = torch.from_numpy(rng.choice(dh.n, 40, replace=False)).cuda()
        a[rows] = float("nan") if k != "scale" else float("inf")
    ctx = gpu_path.context()
    ctx.upload(dh)
    cam = sc.cameras[0]
    img = ctx.render([cam], ctx.select_cut([cam]))
    torch.cuda.synchronize()
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    assert st["device_flags"] == 0
    assert torch.isfinite(img).all()


def test_a_device_wait_that_gives_up_is_flagged_and_the_context_stays_usable():
    import torch
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    ctx = gpu_path.context()
    h3dgs.h3dgs_debug_wait_timeout(ctx.ctx, 2000)
    torch.cuda.synchronize()
    assert h3dgs.h3dgs_get_stats(ctx.ctx)["device_flags"] & 0x8
    cam = sc.cameras[0]
    img = ctx.render([cam], ctx.select_cut([cam]))
    torch.cuda.synchronize()
    assert h3dgs.h3dgs_get_stats(ctx.ctx)["device_flags"] == 0
    fr = oracle.render(cam, h, oracle.Opts())
    im = img.view(3, cam.height, cam.width).cpu().numpy()
    assert np.abs(im - fr.image).max(axis=0)[~fr.ambiguous].max() <= 2e-3
