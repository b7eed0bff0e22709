"""Runs the CUDA path through the C ABI and collects everything the parity tests compare."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from paper_2406_12080_b300 import h3dgs


@dataclass
class GpuFrame:
    cut_ids: np.ndarray
    cut_t: np.ndarray
    offsets: np.ndarray
    images: list
    rec: np.ndarray = None
    rect: np.ndarray = None
    rgb: np.ndarray = None
    T_final: np.ndarray = None
    n_contrib: np.ndarray = None
    stats: dict = None


_ctx = None


def context():
    global _ctx
    import torch
    if _ctx is None:
        _ctx = h3dgs.Context(torch.cuda.current_device())
    return _ctx


def upload(hier):
    ctx = context()
    dh = h3dgs.DeviceHierarchy.from_arrays(hier)
    ctx.upload(dh)
    return dh


def opts_from(o, chunk=None) -> h3dgs.h3dgs_render_opts:
    """Library options equal to the oracle's Opts `o` (plus the blend chunk, which the oracle lacks)."""
    kw = {} if chunk is None else {"blend_chunk": chunk}
    return h3dgs.default_opts(tile_w=o.tile_w, tile_h=o.tile_h, lowpass=o.lowpass, alpha_clamp=o.alpha_clamp,
                              alpha_floor=o.alpha_floor, t_min=o.t_min, aa_compensate=o.aa_compensate,
                              interpolate=o.interpolate, bg=o.bg, **kw)


def run(hier_dev, cams, oopts, debug=True, capacity=None, chunk=None) -> GpuFrame:
    import torch
    ctx = context()
    cut = ctx.select_cut(cams, capacity)
    ids, t, offs = cut
    opts = opts_from(oopts, chunk)
    images = ctx.render(cams, cut, opts, save_for_backward=1)
    torch.cuda.synchronize()
    fr = GpuFrame(ids.cpu().numpy(), t.cpu().numpy(), offs.cpu().numpy(),
                  [im.cpu().numpy() for im in ctx.split_images(images, cams)])
    if debug:
        m = len(fr.cut_ids)
        fr.rec, fr.rect, fr.rgb = h3dgs.h3dgs_debug_splats(ctx.ctx, m)
        npix = sum(c.width * c.height for c in cams)
        fr.T_final, fr.n_contrib = h3dgs.h3dgs_debug_pixel_state(ctx.ctx, npix)
        fr.stats = h3dgs.h3dgs_get_stats(ctx.ctx)
        assert fr.stats["device_flags"] & 0x8 == 0, "a bounded inter-block wait timed out"
        assert fr.stats["device_flags"] & 0x80 == 0, h3dgs.h3dgs_last_error(ctx.ctx)   # checked build only
    fr._images_dev = images
    fr._cut = cut
    return fr


def tile_lists(cam_index: int, n_tiles: int):
    return h3dgs.h3dgs_debug_tile_lists(context().ctx, cam_index, n_tiles)
