"""Pins of the oracle's expected-depth channel (appendix, depth regularisation: the splat colour
replaced by the view depth of its mean) and of the exposure affine (appendix, exposure
optimisation: out = E [C | 1]) against facts fixed independently: the telescoping sum of a scene at
one depth, the affine map applied by numpy, and central finite differences of the adjoint."""
import numpy as np

import oracle
from paper_2406_12080_b300 import synth
from tests import scenes
from tests.test_oracle_pins import _fd_scene


def test_depth_of_a_scene_at_one_depth_telescopes():
    """With every splat at view depth z0, sum_i T_i alpha_i z0 = z0 (1 - T_final)."""
    rng = np.random.default_rng(4)
    n = 300
    mean = np.column_stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.0, 1.0, n), np.full(n, 4.0)])
    scale = np.exp(rng.normal(-2.6, 0.4, size=(n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.uniform(0.3, 0.95, n)
    h = oracle.build_tree(scenes.leaves_from(mean, scale, q, op))
    for tau in (0.0, 4.0, 12.0):
        cam = scenes.axis_camera(96, 64, 80.0, tau=tau)
        fr = oracle.render(cam, h, oracle.Opts())
        assert (1 - fr.T_final).max() > 0.5
        np.testing.assert_allclose(fr.depth, 4.0 * (1.0 - fr.T_final), rtol=0, atol=1e-12)


def test_depth_of_a_single_splat_at_its_centre():
    """One Gaussian on the optical axis: at the centre pixel, depth = alpha z with alpha the clamped
    compensated opacity (G = 1 there)."""
    lv = scenes.leaves_from([[0.0, 0.0, 3.0]], [[0.05, 0.05, 0.05]], [[1.0, 0.0, 0.0, 0.0]], [0.8])
    h = oracle.build_tree(lv)
    cam = scenes.axis_camera(32, 32, 40.0, cx=16.5, cy=16.5)   # the mean projects on pixel (16, 16)'s centre
    fr = oracle.render(cam, h, oracle.Opts())
    s = 40.0 * float(np.float32(0.05)) / 3.0          # the stored (fp32) scale, projected
    comp = np.sqrt(s ** 4 / (s ** 2 + float(np.float32(0.3))) ** 2)
    alpha = min(0.99, float(np.float32(0.8)) * comp)
    assert abs(fr.depth[16, 16] - alpha * 3.0) < 1e-12


def test_exposure_is_the_affine_map_of_the_rendered_colour():
    sc, h = scenes.tiny()
    cam = sc.cameras[0]
    opts = oracle.Opts(bg=(0.2, 0.1, 0.4))
    base = oracle.render(cam, h, opts)
    ident = np.hstack([np.eye(3), np.zeros((3, 1))])
    np.testing.assert_array_equal(oracle.render(cam, h, opts, exposure=ident).image, base.image)
    E = (ident + np.random.default_rng(5).normal(0, 0.2, size=(3, 4))).astype(np.float32)
    fr = oracle.render(cam, h, opts, exposure=E)
    want = np.einsum("ck,khw->chw", E[:, :3].astype(np.float64), base.image) + E[:, 3, None, None]
    np.testing.assert_allclose(fr.image, want, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(fr.depth, base.depth)


def test_backward_with_depth_and_exposure_matches_finite_differences():
    h, cam = _fd_scene()
    opts = oracle.Opts()
    a64 = oracle.Attrs64.of(h)
    rng = np.random.default_rng(6)
    E = (np.hstack([np.eye(3), np.zeros((3, 1))]) + rng.normal(0, 0.15, size=(3, 4))).astype(np.float32)
    fr = oracle.render(cam, h, opts, a64, exposure=E)
    w = rng.normal(size=fr.image.shape)
    wd = rng.normal(size=fr.depth.shape) * 0.3
    g = oracle.backward(cam, h, fr, w, opts, a64, dL_ddepth=wd, exposure=E)
    g0 = oracle.backward(cam, h, fr, w, opts, a64, exposure=E)
    assert np.abs(g[:, :3] - g0[:, :3]).max() > 1e-3 * np.abs(g0[:, :3]).max()   # depth reaches the means
    touched = np.unique(np.concatenate([fr.ids, h.parent[fr.ids][h.parent[fr.ids] >= 0]]))
    f = lambda: oracle.weighted_image_sum(cam, h, fr, w, opts, a64, w_depth=wd, exposure=E)
    gmax = np.abs(g).max()
    checked = skipped = 0
    for node in rng.choice(touched, size=min(len(touched), 16), replace=False):
        for name, c0, cols in (("mean", 0, range(3)), ("opacity", 10, range(1)), ("scale", 3, range(3)),
                               ("sh", 11, (0, 1, 2))):
            arr = getattr(a64, name)
            flat = arr.reshape(arr.shape[0], -1)
            for j in cols:
                theta = flat[node, j]
                step = 1e-6 * max(abs(theta), 0.05)
                flat[node, j] = theta + step
                fp = f()
                flat[node, j] = theta - step
                fm = f()
                flat[node, j] = theta
                f0 = f()
                fwd, bwd = (fp - f0) / step, (f0 - fm) / step
                if abs(fwd - bwd) > 0.1 * max(abs(fwd), abs(bwd), 1e-6 * gmax):
                    skipped += 1
                    continue
                fd = (fp - fm) / (2 * step)
                an = g[node, c0 + j]
                assert abs(fd - an) <= 1e-4 * max(abs(fd), abs(an)) + 1e-7 * gmax, (name, node, j, fd, an)
                checked += 1
    assert checked > 100 and skipped < 0.15 * checked
