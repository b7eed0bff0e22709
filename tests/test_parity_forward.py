"""Parity of the CUDA forward path (cut, interpolation, splats, tile lists, image) with the oracle.

Bars: bit-exact for the cut (ids and t), the interpolated fp32 attributes, the splat records
(the decision track), tile rectangles and per-tile lists; images within 2e-3 max abs per channel
on every pixel whose per-pixel decisions are unambiguous in fp32 (the oracle flags those within
a 1e-5 relative band of the alpha floor or the transmittance stop), and the flagged fraction
below 2e-4 (measured: at most 5e-5 on the test scenes).  Full-size parity runs the 1M-leaf street corridor at 1920x1080.
"""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import synth
from tests import gpu_path, scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()


def _compare(cam, h, dh, opts, cams_index=0, chunk=None):
    ofr = oracle.render(cam, h, opts)
    g = gpu_path.run(dh, [cam], opts, chunk=chunk)
    # a1/a2: cut ids and weights bit-exact
    np.testing.assert_array_equal(g.cut_ids, ofr.ids)
    np.testing.assert_array_equal(g.cut_t.view(np.uint32), ofr.t.view(np.uint32))
    # a4: splat records and rectangles (fp32 decision track) bit-exact
    np.testing.assert_array_equal(g.rect, ofr.rect)
    vis = ofr.rect[:, 0] >= 0
    np.testing.assert_array_equal(g.rec[vis].view(np.uint32), ofr.rec32[vis].view(np.uint32))
    # colour (value track): fp32 vs fp64
    np.testing.assert_allclose(g.rgb[vis], ofr.val64[vis, 9:12], atol=2e-5, rtol=1e-5)
    # a5/a6: per-tile lists bit-exact (node ids in list order)
    TX, TY = oracle.tiles(cam, opts)
    ranges, ids = gpu_path.tile_lists(cams_index, TX * TY)
    np.testing.assert_array_equal(ranges[:, 1] - ranges[:, 0], ofr.ranges[:, 1] - ofr.ranges[:, 0])
    np.testing.assert_array_equal(ids, ofr.ids[ofr.lists])
    # a7: image and per-pixel state
    amb = ofr.ambiguous
    img = g.images[0]
    err = np.abs(img - ofr.image).max(axis=0)
    assert amb.mean() < 2e-4
    assert err[~amb].max() <= IMG_TOL, err[~amb].max()
    nc = g.n_contrib.reshape(cam.height, cam.width)
    np.testing.assert_array_equal(nc[~amb], ofr.n_contrib[~amb])
    np.testing.assert_allclose(g.T_final.reshape(cam.height, cam.width)[~amb], ofr.T_final[~amb], atol=2e-4, rtol=1e-3)
    return ofr, g


@pytest.mark.parametrize("tau", [0.0, 2.0, 6.0, 15.0, 80.0, float("inf")])
def test_tiny_scene_all_stages(tau):
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], tau)
    ofr, g = _compare(cam, h, dh, oracle.Opts())
    assert g.stats["n_cut"] == len(ofr.ids)
    assert g.stats["n_pairs"] == len(ofr.lists)



@pytest.mark.parametrize("seed", range(10))
def test_random_scenes_and_cameras(seed):
    """Every bar of the forward path on seeded random scenes and cameras (one of them sees
    nothing)."""
    h, cam = scenes.random_case(seed)
    dh = gpu_path.upload(h)
    ofr, g = _compare(cam, h, dh, oracle.Opts())
    assert g.stats["n_cut"] == len(ofr.ids) and g.stats["n_pairs"] == len(ofr.lists)

@pytest.mark.parametrize("tw,th", [(8, 8), (32, 8), (8, 32), (16, 8)])
def test_tile_shapes(tw, th):
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    _compare(sc.cameras[0], h, dh, oracle.Opts(tile_w=tw, tile_h=th))


def test_options_interpolation_off_no_compensation_background():
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    _compare(sc.cameras[0], h, dh, oracle.Opts(interpolate=0))
    _compare(sc.cameras[0], h, dh, oracle.Opts(aa_compensate=0, lowpass=0.1, bg=(0.2, 0.5, 1.0)))


def test_ragged_image_and_offcentre_camera():
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    c = sc.cameras[0]
    cam = synth.Camera(c.R, c.T, 180.0, 200.0, 61.3, 47.9, 133, 97, 5.0)
    _compare(cam, h, dh, oracle.Opts())


def test_camera_inside_the_scene():
    """Camera inside the root box: eps(root) = inf, parents with inf granularity give t = 0."""
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    cam = synth.look_camera([5.0, 5.0, 5.0], [0.3, 0.2, 1.0], [0, -1, 0], 160, 120, 70.0, 6.0)
    _compare(cam, h, dh, oracle.Opts())


def test_single_node_hierarchy_and_everything_culled():
    lv = scenes.leaves_from([[0, 0, 5.0]], [[0.2, 0.1, 0.3]], [[0.9, 0.1, 0.2, 0.3]], [0.7])
    h = oracle.build_tree(lv)
    dh = gpu_path.upload(h)
    cam = scenes.axis_camera(40, 30, 50.0)
    _compare(cam, h, dh, oracle.Opts())
    behind = scenes.axis_camera(40, 30, 50.0, pos=(0, 0, 10.0))   # the Gaussian is behind the camera
    ofr, g = _compare(behind, h, dh, oracle.Opts())
    assert g.stats["n_visible"] == 0 and np.all(g.images[0] == 0)


def test_multi_camera_batch_matches_single_views():
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    base = sc.cameras[0]
    cams = [synth.with_tau(base, 6.0),
            synth.look_camera([5, 5, -12.0], [0.1, 0, 1], [0, -1, 0], 200, 150, 60.0, 3.0),
            synth.look_camera([-8, 5, 5.0], [1, 0, 0.05], [0, -1, 0], 96, 128, 75.0, 15.0)]
    g = gpu_path.run(dh, cams, oracle.Opts())
    for k, cam in enumerate(cams):
        ofr = oracle.render(cam, h, oracle.Opts())
        lo, hi = g.offsets[k], g.offsets[k + 1]
        np.testing.assert_array_equal(g.cut_ids[lo:hi], ofr.ids)
        np.testing.assert_array_equal(g.cut_t[lo:hi].view(np.uint32), ofr.t.view(np.uint32))
        err = np.abs(g.images[k] - ofr.image).max(axis=0)
        assert err[~ofr.ambiguous].max() <= IMG_TOL
        TX, TY = oracle.tiles(cam, oracle.Opts())
        ranges, ids = gpu_path.tile_lists(k, TX * TY)
        np.testing.assert_array_equal(ranges[:, 1] - ranges[:, 0], ofr.ranges[:, 1] - ofr.ranges[:, 0])
        np.testing.assert_array_equal(ids, ofr.ids[ofr.lists])


def test_interpolate_export_bit_exact():
    from paper_2406_12080_b300 import h3dgs
    import torch
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    cam = sc.cameras[0]
    ctx = gpu_path.context()
    ids, t, offs = ctx.select_cut([cam])
    M = int(ids.shape[0])
    out = torch.empty((h3dgs.NINTERP, M), dtype=torch.float32, device="cuda")
    h3dgs.h3dgs_interpolate(ctx.ctx, [cam], ids, t, offs, 1, out, M)
    o32, o64 = oracle.interpolate(h, ids.cpu().numpy(), t.cpu().numpy())
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), o32.view(np.uint32))
    np.testing.assert_allclose(out.cpu().numpy(), o64, atol=1e-6, rtol=1e-6)


@pytest.mark.parametrize("chunk", [64, 100, 150])
def test_split_tiles_small_chunks(chunk):
    """Tile lists longer than the blend chunk are blended by several CTAs and recombined."""
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    ofr, g = _compare(synth.with_tau(sc.cameras[0], 2.0), h, dh, oracle.Opts(), chunk=chunk)
    lengths = ofr.ranges[:, 1] - ofr.ranges[:, 0]
    expected_items = int(np.sum(np.where(lengths <= chunk, 1, (lengths + chunk - 1) // chunk)))
    assert g.stats["n_items"] == expected_items


@pytest.mark.parametrize("tau,chunk", [(0.0, None), (3.0, None), (6.0, None), (15.0, None), (6.0, 64), (6.0, 4096)])
def test_street_corridor_full_size(tau, chunk):
    """1M leaves (2M nodes) at 1920x1080: the workload the benchmark times."""
    sc, h = scenes.corridor()
    dh = gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], tau)
    _compare(cam, h, dh, oracle.Opts(), chunk=chunk)


def test_one_tile_with_twenty_thousand_splats():
    """A tile list longer than 16384 entries takes the global-scratch sort path and many blend chunks."""
    rng = np.random.default_rng(21)
    n, f = 20000, 100.0
    z = rng.uniform(5.0, 50.0, n)
    u = rng.uniform(18.0, 30.0, n)
    v = rng.uniform(18.0, 30.0, n)
    mean = np.stack([(u - 32.0) * z / f, (v - 32.0) * z / f, z], 1)
    scale = (0.3 * z / f)[:, None] * np.exp(rng.normal(0, 0.2, (n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.uniform(0.02, 0.2, n)
    lv = scenes.leaves_from(mean, scale, q, op, rng.normal(0, 0.3, (n, 48)))
    h = oracle.build_tree(lv)
    dh = gpu_path.upload(h)
    cam = scenes.axis_camera(64, 64, f, tau=0.0)
    ofr, g = _compare(cam, h, dh, oracle.Opts())
    lengths = ofr.ranges[:, 1] - ofr.ranges[:, 0]
    assert lengths.max() > 16384



@pytest.mark.parametrize("which,chunk", [("tiny", 64), ("tiny", 100), ("full_size_corridor", 64),
                                         ("full_size_corridor", None)])
def test_middle_chunk_shortcut_and_counting(which, chunk):
    """Consumers of middle chunks take the producer's local walk times T_in at the pixels that cannot stop
    inside the chunk.  While counting (profiling level 2) every consumer walks all its pixels and then
    takes the same values, so the outputs are bit-identical with and without counting; in the checked
    build the counting kernel also verifies that each such walk did not stop and ended on the producer's
    last contributor (bit 7 of the device flags, asserted clear by gpu_path.run)."""
    from paper_2406_12080_b300 import h3dgs
    sc, h = scenes.tiny() if which == "tiny" else scenes.corridor()
    dh = gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], 2.0 if which == "tiny" else 6.0)
    ctx = gpu_path.context()
    runs = []
    for prof in (0, 2):
        h3dgs.h3dgs_set_profiling(ctx.ctx, prof)
        try:
            g = gpu_path.run(dh, [cam], oracle.Opts(), chunk=chunk)
        finally:
            h3dgs.h3dgs_set_profiling(ctx.ctx, 0)
        runs.append(g)
    a, b = runs
    ranges, _ = gpu_path.tile_lists(0, int(b.stats["n_tiles"]))
    lens = ranges[:, 1] - ranges[:, 0]
    c = chunk or 320
    middle = bool(np.any(lens > 2 * c))       # tiles of three or more chunks
    assert middle or chunk != 64
    assert (b.stats["n_evals_tpass"] > 0) == middle
    np.testing.assert_array_equal(a.images[0].view(np.uint32), b.images[0].view(np.uint32))
    np.testing.assert_array_equal(a.T_final.view(np.uint32), b.T_final.view(np.uint32))
    np.testing.assert_array_equal(a.n_contrib, b.n_contrib)


@pytest.mark.parametrize("which", ["single", "batch"])
def test_reserved_capacities_render_the_same_frame(which):
    """With fixed capacities (h3dgs_reserve) one launch clears the frame's counters and workspaces and
    sets up the cameras, and the sorts and the plan use pre-zeroed workspaces; the frame must be the one
    the unreserved path renders, bit for bit (images, per-pixel state, tile lists)."""
    from paper_2406_12080_b300 import h3dgs
    sc, h = scenes.tiny()
    dh = gpu_path.upload(h)
    base = sc.cameras[0]
    cams = [synth.with_tau(base, 2.0)] if which == "single" else [
        synth.with_tau(base, 6.0),
        synth.look_camera([5, 5, -12.0], [0.1, 0, 1], [0, -1, 0], 200, 150, 60.0, 3.0),
        synth.look_camera([-8, 5, 5.0], [1, 0, 0.05], [0, -1, 0], 96, 128, 75.0, 15.0)]
    o = oracle.Opts()
    a = gpu_path.run(dh, cams, o, chunk=64)
    tiles = [int(np.prod(oracle.tiles(c, o))) for c in cams]
    la = [gpu_path.tile_lists(k, n) for k, n in enumerate(tiles)]
    ctx = gpu_path.context()
    try:
        h3dgs.h3dgs_reserve(ctx.ctx, len(a.cut_ids) + 64, 4 * int(a.stats["n_pairs"]) + 1024)
        b = gpu_path.run(dh, cams, o, chunk=64)
        lb = [gpu_path.tile_lists(k, n) for k, n in enumerate(tiles)]
    finally:
        h3dgs.h3dgs_reserve(ctx.ctx, 0, 0)
    assert b.stats["device_flags"] == 0
    for ia, ib in zip(a.images, b.images):
        np.testing.assert_array_equal(ia.view(np.uint32), ib.view(np.uint32))
    np.testing.assert_array_equal(a.T_final.view(np.uint32), b.T_final.view(np.uint32))
    np.testing.assert_array_equal(a.n_contrib, b.n_contrib)
    for (ra, ia), (rb, ib) in zip(la, lb):
        np.testing.assert_array_equal(ra, rb)
        np.testing.assert_array_equal(ia, ib)


def test_automatic_chunk_splits_a_light_frame_at_320():
    """The default (automatic) blend chunk of the 1080p corridor frame (mean list length 165, below 450)
    is 320: the plan cuts each list of L > 320 entries into ceil(L / 320) chunks."""
    sc, h = scenes.corridor()
    dh = gpu_path.upload(h)
    cam = synth.with_tau(sc.cameras[0], 6.0)
    g = gpu_path.run(dh, [cam], oracle.Opts())          # default options: the automatic chunk
    TX, TY = oracle.tiles(cam, oracle.Opts())
    ranges, _ = gpu_path.tile_lists(0, TX * TY)
    lens = ranges[:, 1] - ranges[:, 0]
    want = int(np.sum(np.where(lens <= 320, 1, (lens + 319) // 320)))
    assert g.stats["n_items"] == want > TX * TY
