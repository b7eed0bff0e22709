"""The blend's profiling counters (profiling level 2): the counting variant renders the same image,
and the counts respect bounds that any correct blend satisfies.

* Every main-pass evaluation is one (pixel, list entry) pair of the pixel's tile, each pair taken at
  most once, so the count is at most the sum over the image's pixels of their tile's list length
  (the oracle's lists).
* Evaluations of splats with an interpolated parent (t != 0, where the transition alpha of Eq. alphap
  is evaluated too) are a subset of the main-pass ones, and there are none with interpolation off.
* The middle chunks' producer walks (counted apart) exist only for split tiles: none when the chunk
  exceeds every list.
"""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs
from tests import gpu_path, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _counted(ctx, cam, cut, opts):
    import torch
    plain = ctx.render([cam], cut, opts).clone()
    h3dgs.h3dgs_set_profiling(ctx.ctx, 2)
    try:
        counted = ctx.render([cam], cut, opts)
        torch.cuda.synchronize()
        st = h3dgs.h3dgs_get_stats(ctx.ctx)
    finally:
        h3dgs.h3dgs_set_profiling(ctx.ctx, 0)
    assert torch.equal(plain, counted)
    return st


def _pixel_list_sum(cam, ofr, o):
    TX, TY = oracle.tiles(cam, o)
    lens = (ofr.ranges[:, 1] - ofr.ranges[:, 0]).reshape(TY, TX).astype(np.int64)
    ty = np.arange(cam.height) // o.tile_h
    tx = np.arange(cam.width) // o.tile_w
    return int(lens[ty[:, None], tx[None, :]].sum())


@pytest.mark.parametrize("chunk", [64, 65536])
def test_counts_are_bounded_and_do_not_change_the_image(chunk):
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    ctx = gpu_path.context()
    cam = sc.cameras[0]
    o = oracle.Opts()
    ofr = oracle.render(cam, h, o)
    cut = ctx.select_cut([cam])
    st = _counted(ctx, cam, cut, gpu_path.opts_from(o, chunk))
    assert 0 < st["n_evals"] <= _pixel_list_sum(cam, ofr, o)
    assert 0 <= st["n_evals_interp"] <= st["n_evals"]
    if np.any(ofr.t != 0):
        assert st["n_evals_interp"] > 0
    lens = ofr.ranges[:, 1] - ofr.ranges[:, 0]
    if lens.max() <= chunk:
        assert st["n_evals_tpass"] == 0


def test_no_interpolated_evaluations_without_interpolation():
    sc, h = scenes.tiny()
    gpu_path.upload(h)
    ctx = gpu_path.context()
    cam = sc.cameras[0]
    o = oracle.Opts(interpolate=0)
    cut = ctx.select_cut([cam])
    st = _counted(ctx, cam, cut, gpu_path.opts_from(o))
    assert st["n_evals"] > 0
    assert st["n_evals_interp"] == 0
