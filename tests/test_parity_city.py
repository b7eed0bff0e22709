"""The large-scene workload at full size: 50M leaves in 20 x 20 chunks of 50 m, one hierarchy per chunk
joined by a top tree over the chunk roots (h3dgs_build_hierarchy_chunked), about 100M nodes.

The oracle cannot build the whole scene in a test's time, so parity is checked where the oracle can
work one chunk at a time: for sampled chunks the oracle builds the chunk's hierarchy from the chunk's
leaves alone, and the device's nodes of that chunk must match it (topology, boxes bit-exact, attributes
within fp32 rounding), and the device cut of full-size frames must hold exactly the chunk nodes the
oracle's cut rule selects, with identical weights (every chunk node but the root has its parent inside
the chunk, so its decision is local).  Properties that hold at any size are checked on the whole
scene: the cut is an antichain meeting every root-to-leaf path exactly once, and the images, final
transmittances and contributor counts are in range.

The image is compared with the oracle on the 4 x 4 chunks around pose 0 of the camera loop (2M
leaves, about 4M nodes): the oracle builds each chunk and consolidates them under a top tree
(oracle.consolidate), the device's chunked build of the same leaves must equal that hierarchy, and the
frame of pose 0 rendered from the oracle's hierarchy must match the oracle's render (cut, weights,
splat records and tile lists bit-exact; image within 2e-3 on unambiguous pixels)."""
import functools

import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import h3dgs, synth
from tests import gpu_path, scenes

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
GRID, PER = 20, 125_000
CHUNKS = (0, 137, 399)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def _city():
    import torch
    ctx = gpu_path.context()
    leaves, off = scenes.city_device(ctx, GRID, PER)
    dh = ctx.build_chunked(leaves, off)
    del leaves
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return dh


def _chunk_nodes(dh, c):
    """Global node ids of chunk c's local nodes 0 .. 2 PER - 2 (local 0 = the chunk root)."""
    n_top = 2 * GRID * GRID - 1
    base = n_top + c * (2 * PER - 2)
    cs = dh.child_start[:n_top].cpu().numpy()
    root = int(np.nonzero(cs == base)[0][0])
    return np.concatenate([[root], base + np.arange(2 * PER - 2)]), base


def test_chunk_hierarchies_equal_the_oracle_build():
    dh = _city()
    assert dh.n == 2 * GRID * GRID * PER - 1
    for c in CHUNKS:
        ho = oracle.build_tree(synth.city_chunk_leaves(2, c % GRID, c // GRID, PER))
        g, base = _chunk_nodes(dh, c)
        gid = lambda local: np.where(local < 0, -1, np.where(local == 0, g[0], base + local - 1))
        par = dh.parent[g].cpu().numpy()
        np.testing.assert_array_equal(par[1:], gid(ho.parent[1:]))
        cs = dh.child_start[g].cpu().numpy()
        np.testing.assert_array_equal(cs, gid(ho.child_start))
        np.testing.assert_array_equal(dh.child_count[g].cpu().numpy(), ho.child_count)
        for k in ("box_min", "box_max"):
            np.testing.assert_array_equal(getattr(dh, k)[g].cpu().numpy(), getattr(ho, k), err_msg=k)
        np.testing.assert_allclose(dh.mean[g].cpu().numpy(), ho.mean, rtol=1e-6, atol=1e-5)
        np.testing.assert_allclose(dh.opacity[g].cpu().numpy(), ho.opacity, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(dh.sh[g].cpu().numpy(), ho.sh, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("pose", [0, 97, 200])
def test_full_size_frame_cut_and_render(pose):
    import torch
    dh = _city()
    ctx = gpu_path.context()
    ctx.upload(dh)
    cam = synth.city_path(2, 256)[pose]
    cut = ctx.select_cut([cam], dh.n)   # the scan (default mode)
    scan_read = h3dgs.h3dgs_get_stats(ctx.ctx)["n_cut_visited"]
    ids, t, _ = cut
    ids_h, t_h = ids.cpu().numpy(), t.cpu().numpy()
    # the root-down traversal selects the same nodes with the same weights, reading far fewer records
    h3dgs.h3dgs_set_cut_mode(ctx.ctx, 2)
    ids_s, t_s, _ = ctx.select_cut([cam], dh.n)
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    h3dgs.h3dgs_set_cut_mode(ctx.ctx, 0)
    assert st["n_cut_visited"] < dh.n // 2 and st["device_flags"] & 0xC == 0
    # the scan skips the far chunks' deep rows and still reads every node the traversal visits
    assert st["n_cut_visited"] <= scan_read < 0.8 * dh.n   # 61% read on average over the loop
    np.testing.assert_array_equal(ids_s.cpu().numpy(), ids_h)
    np.testing.assert_array_equal(t_s.cpu().numpy().view(np.uint32), t_h.view(np.uint32))
    del ids_s, t_s
    assert np.all(np.diff(ids_h) > 0)
    assert np.all((t_h >= 0) & (t_h <= 1))
    # antichain meeting every root-to-leaf path once, level by level (parents precede children)
    parent = dh.parent.cpu().numpy()
    cstart = dh.child_start.cpu().numpy()
    ccount = dh.child_count.cpu().numpy()
    assert set(np.unique(ccount)) <= {0, 2}
    in_cut = np.zeros(dh.n, bool)
    in_cut[ids_h] = True
    covered = in_cut.copy()    # some node on the path from the root down to v (inclusive) is in the cut
    above = np.zeros(dh.n, bool)
    frontier = np.array([0])
    while len(frontier):
        kids = frontier[ccount[frontier] > 0]
        ch = (cstart[kids][:, None] + np.arange(2)[None, :]).ravel()
        assert np.all(parent[ch] == np.repeat(kids, 2))
        above[ch] = covered[parent[ch]]
        covered[ch] |= covered[parent[ch]]
        frontier = ch
    assert not np.any(in_cut & above), "a cut node has a cut ancestor"
    assert np.all(covered[ccount == 0]), "a leaf is not covered by the cut"
    # the sampled chunks: the oracle's cut rule on its own chunk build
    for c in CHUNKS:
        ho = oracle.build_tree(synth.city_chunk_leaves(2, c % GRID, c // GRID, PER))
        oid, ot = oracle.select_cut(cam, ho, 1)
        keep = oid > 0
        g, base = _chunk_nodes(dh, c)
        want = base + oid[keep] - 1
        lo, hi = base, base + 2 * PER - 2
        sel = (ids_h >= lo) & (ids_h < hi)
        np.testing.assert_array_equal(ids_h[sel], want)
        np.testing.assert_array_equal(t_h[sel].view(np.uint32), ot[keep].view(np.uint32))
    # render: values in range
    images = ctx.render([cam], cut, save_for_backward=0)
    torch.cuda.synchronize()
    st = h3dgs.h3dgs_get_stats(ctx.ctx)
    assert st["device_flags"] == 0
    im = images.cpu().numpy()
    assert np.all(np.isfinite(im)) and im.min() >= 0
    npix = cam.width * cam.height
    Tf, nc = h3dgs.h3dgs_debug_pixel_state(ctx.ctx, npix)
    assert np.all((Tf >= 0) & (Tf <= 1)) and np.all(nc >= 0)
    assert st["n_cut"] == len(ids_h) and st["n_visible"] > 0
    # the automatic blend chunk: a frame whose mean list length is above 450 splits no tile list
    assert st["n_pairs"] > 450 * st["n_tiles"]
    assert st["n_items"] == st["n_tiles"]


# ---------------------------------------------------------------- 16-chunk neighbourhood of pose 0

def _neighbourhood():
    """The 4 x 4 chunks around the camera of pose 0: the camera in the second row and column from the
    block's back edge along its viewing direction."""
    cam = synth.city_path(2, 256)[0]
    pos, fwd = synth.city_poses(2, 256)[0]
    cx, cy = int(pos[0] // 50.0), int(pos[1] // 50.0)
    x0 = cx - 1 if fwd[0] >= 0 else cx - 2
    y0 = cy - 1 if fwd[1] >= 0 else cy - 2
    x0, y0 = min(max(x0, 0), GRID - 4), min(max(y0, 0), GRID - 4)
    return cam, [(x, y) for y in range(y0, y0 + 4) for x in range(x0, x0 + 4)]


@functools.lru_cache(maxsize=None)
def _neighbourhood_oracle():
    cam, cells = _neighbourhood()
    leaves = [synth.city_chunk_leaves(2, x, y, PER) for x, y in cells]
    return cam, leaves, oracle.consolidate([oracle.build_tree(lv) for lv in leaves])


def test_neighbourhood_consolidation_equals_the_oracle():
    import torch
    cam, leaves, ho = _neighbourhood_oracle()
    ctx = gpu_path.context()
    dev = {k: torch.from_numpy(np.ascontiguousarray(np.concatenate([getattr(lv, k) for lv in leaves]))).cuda()
           for k in ("mean", "scale", "rot", "opacity", "sh")}
    off = np.arange(len(leaves) + 1, dtype=np.int64) * PER
    dh = ctx.build_chunked(dev, off)
    torch.cuda.synchronize()
    assert dh.n == ho.n
    for k in ("parent", "child_start", "child_count", "box_min", "box_max"):
        np.testing.assert_array_equal(getattr(dh, k).cpu().numpy(), getattr(ho, k), err_msg=k)
    np.testing.assert_allclose(dh.mean.cpu().numpy(), ho.mean, rtol=1e-6, atol=2e-5)
    np.testing.assert_allclose(dh.opacity.cpu().numpy(), ho.opacity, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(dh.sh.cpu().numpy(), ho.sh, rtol=1e-5, atol=1e-6)
    s_d = dh.scale.cpu().numpy()
    np.testing.assert_allclose(s_d, ho.scale, rtol=1e-4, atol=1e-6)


def test_neighbourhood_frame_matches_the_oracle():
    from tests.test_parity_forward import _compare
    cam, _, ho = _neighbourhood_oracle()
    dh = gpu_path.upload(ho)
    ofr, g = _compare(cam, ho, dh, oracle.Opts())
    assert len(ofr.ids) > 100_000 and np.sum(ofr.t > 0) > 10_000
    assert g.stats["n_pairs"] == len(ofr.lists)


# ---------------------------------------------------------------- C4: 32 mixed-resolution views at once

def test_c4_batch_of_32_views_equals_single_views():
    """32 cameras on the city loop, 8 each at 1280x720, 1920x1080, 2560x1440 and 3840x2160 with tau
    cycling over 3, 6, 15, in one cut + render + adjoint: every image equals the camera rendered alone
    bit for bit, and the node gradients equal the sum of the per-camera adjoints (fp32 reductions in
    another order: the per-element bar of tests/test_parity_backward.py).  The blend chunk is explicit:
    the automatic one depends on the frame's total work (the batch would split no list, a single view
    at 320), and chunked walks reassociate T."""
    import torch
    dh = _city()
    ctx = gpu_path.context()
    ctx.upload(dh)
    cams = synth.city_views(2, 32)
    N = dh.n
    ids1 = torch.empty(N, dtype=torch.int32, device="cuda")
    t1 = torch.empty(N, dtype=torch.float32, device="cuda")
    offs1 = torch.empty(2, dtype=torch.int64, device="cuda")
    sizes = [h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids1, t1, offs1, N) for c in cams]
    cap = int(sum(sizes)) + 1024
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    t = torch.empty(cap, dtype=torch.float32, device="cuda")
    offs = torch.empty(len(cams) + 1, dtype=torch.int64, device="cuda")
    assert h3dgs.h3dgs_select_cut(ctx.ctx, cams, ids, t, offs, cap) == sum(sizes)
    npix = [3 * c.width * c.height for c in cams]
    poff = np.concatenate([[0], np.cumsum(npix)])
    opts = h3dgs.default_opts(blend_chunk=320)
    img_b = torch.empty(int(poff[-1]), dtype=torch.float32, device="cuda")
    h3dgs.h3dgs_render(ctx.ctx, cams, ids, t, offs, opts, img_b, 1)
    dl = torch.randn(int(poff[-1]), generator=torch.Generator(device="cuda").manual_seed(5), device="cuda")
    keys = ("mean", "scale", "rot", "opacity", "sh")
    gb = {k: torch.zeros_like(getattr(dh, k)) for k in keys}
    h3dgs.h3dgs_render_backward(ctx.ctx, dl, gb, 1)
    torch.cuda.synchronize()
    assert h3dgs.h3dgs_get_stats(ctx.ctx)["device_flags"] == 0
    gv = {k: torch.zeros_like(getattr(dh, k)) for k in keys}
    img_v = torch.empty_like(img_b)
    for k, c in enumerate(cams):
        lo, hi = int(poff[k]), int(poff[k + 1])
        h3dgs.h3dgs_select_cut(ctx.ctx, [c], ids1, t1, offs1, N)
        h3dgs.h3dgs_render(ctx.ctx, [c], ids1, t1, offs1, opts, img_v[lo:hi], 1)
        h3dgs.h3dgs_render_backward(ctx.ctx, dl[lo:hi], gv, 1)   # accumulates
    torch.cuda.synchronize()
    assert torch.equal(img_b, img_v)
    # the per-element bar, evaluated on the device (tens of millions of touched rows)
    touched = 0
    for k in keys:
        a_all, b_all = gb[k].reshape(N, -1), gv[k].reshape(N, -1)
        scale = b_all.abs().max().item()
        assert scale > 0, k
        excess, d2, b2, tk = 0.0, 0.0, 0.0, 0
        for r0 in range(0, N, 8_000_000):   # row chunks bound the temporaries
            a, b = a_all[r0:r0 + 8_000_000], b_all[r0:r0 + 8_000_000]
            excess = max(excess, ((a - b).abs() - 1e-3 * b.abs()).max().item() / scale)
            d2 += float(((a - b).double() ** 2).sum().item())
            b2 += float((b.double() ** 2).sum().item())
            tk += int((b.abs().amax(1) > 0).sum().item())
        assert excess <= 1e-5, (k, excess)
        assert d2 ** 0.5 <= 1e-3 * b2 ** 0.5, k
        touched = max(touched, tk)
    assert touched > 1_000_000
