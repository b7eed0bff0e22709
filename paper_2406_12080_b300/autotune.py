"""Autotuner for the render's launch shape: screen tile (TW x TH) and blend chunk.

The per-tile work of the blend is heavy-tailed in street scenes, so the best tile shape and the
chunk length at which a tile's list is split across CTAs depend on the view set.  The tuner times
each candidate on the actual cameras and cut (CUDA events on the context's stream, after warm-up)
and keeps the fastest; results are cached in a JSON file keyed by GPU name, resolution class and
camera count.  Images do not depend on the choice beyond fp32 reassociation of T in split tiles.
"""
from __future__ import annotations

import json
import os

from . import h3dgs

TILES = ((16, 16), (32, 8), (16, 8), (8, 32))
CHUNKS = (256, 320, 384, 512, 1024, 65536)
CACHE_PATH = os.environ.get("H3DGS_TUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json"))


def resolution_class(cams) -> str:
    px = sum(c.width * c.height for c in cams)
    return f"{len(cams)}cams_{px // 100000}e5px"


def _key(cams) -> str:
    import torch
    return f"{torch.cuda.get_device_name()}|{resolution_class(cams)}"


def load_cache() -> dict:
    try:
        return json.load(open(CACHE_PATH))
    except Exception:
        return {}


def save_cache(c: dict) -> None:
    tmp = CACHE_PATH + ".tmp"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE_PATH)


def tune(ctx: h3dgs.Context, cams, cut, images, reps: int = 5, use_cache: bool = True, base_opts=None):
    """Returns (opts, table): the fastest render options and the time (ms) of every candidate."""
    import torch
    key = _key(cams)
    cache = load_cache() if use_cache else {}
    if key in cache:
        tw, th, ch = cache[key]["best"]
        return h3dgs.default_opts(tile_w=tw, tile_h=th, blend_chunk=ch), cache[key]["table"]
    ids, t, offs = cut
    carr = h3dgs.camera_array(cams)
    stream = ctx.stream
    table = {}
    best = None
    for tw, th in TILES:
        for ch in CHUNKS:
            opts = h3dgs.default_opts(tile_w=tw, tile_h=th, blend_chunk=ch)
            for _ in range(2):
                h3dgs.h3dgs_render(ctx.ctx, cams, ids, t, offs, opts, images, 0, cam_array=carr)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                h3dgs.h3dgs_render(ctx.ctx, cams, ids, t, offs, opts, images, 0, cam_array=carr)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            table[f"{tw}x{th}/{ch}"] = ms
            if best is None or ms < best[0]:
                best = (ms, tw, th, ch)
    _, tw, th, ch = best
    if use_cache:
        cache[key] = {"best": [tw, th, ch], "table": table}
        save_cache(cache)
    return h3dgs.default_opts(tile_w=tw, tile_h=th, blend_chunk=ch), table
