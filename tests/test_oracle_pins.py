"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper it checks and the independent fact used: a closed
form, a Monte-Carlo estimate, brute force, an invariant, or a textbook routine (scipy).
"""
import functools
import itertools
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle
from paper_2406_12080_b300 import synth
from tests import scenes


def _rotmat(q_wxyz):
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def _cov(scale, q_wxyz):
    R = _rotmat(q_wxyz)
    return R @ np.diag(np.asarray(scale, np.float64) ** 2) @ R.T


def _row(mu, s, q, o, sh=None):
    sh = np.zeros(48) if sh is None else sh
    return np.concatenate([mu, s, q, [o], sh]).astype(np.float64)


def _random_row(rng, scale=None):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    s = np.exp(rng.normal(-1, 0.5, 3)) if scale is None else np.asarray(scale)
    return _row(rng.normal(size=3), s, q, rng.uniform(0.2, 0.9), rng.normal(0, 0.3, 48))


# ------------------------------------------------------------------ spherical harmonics (colour)

def test_sh_basis_orthonormal_and_matches_scipy():
    """Real SH to degree 3: orthonormal on the sphere (Gauss-Legendre x uniform-phi quadrature,
    exact for these polynomials) and equal, up to a sign per function, to scipy's Y_l^m."""
    mu, wmu = np.polynomial.legendre.leggauss(12)
    phis = np.arange(24) * (2 * np.pi / 24)
    B, Bs, w = [], [], []
    for m_, wm in zip(mu, wmu):
        th = math.acos(m_)
        for ph in phis:
            d = (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), m_)
            B.append(oracle.sh_basis(d))
            row = []
            for l in range(4):
                for m in range(-l, l + 1):
                    y = sph_harm_y(l, abs(m), th, ph)
                    row.append(y.real if m == 0 else math.sqrt(2) * (y.real if m > 0 else y.imag))
            Bs.append(row)
            w.append(wm * 2 * np.pi / 24)
    B, Bs, w = np.array(B), np.array(Bs), np.array(w)
    gram = (B * w[:, None]).T @ B
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)
    cross = np.diag((B * w[:, None]).T @ Bs)
    np.testing.assert_allclose(np.abs(cross), 1.0, atol=1e-12)


# ------------------------------------------------------------------ merge (Sec. 4.1, Eq. merge)

def test_ellipsoid_area_closed_forms():
    """The weight area S_i: exact for a sphere (4 pi r^2), within Thomsen's 1.1% of the closed
    form for prolate and oblate spheroids."""
    assert oracle.ellipsoid_area([0.7, 0.7, 0.7]) == pytest.approx(4 * np.pi * 0.49, rel=1e-12)
    for a, c in [(1.0, 3.0), (1.0, 10.0), (2.0, 0.5)]:
        if c > a:   # prolate: S = 2 pi a^2 (1 + c/(a e) asin e)
            e = math.sqrt(1 - a * a / (c * c))
            exact = 2 * np.pi * a * a * (1 + c / (a * e) * math.asin(e))
        else:       # oblate: S = 2 pi a^2 (1 + (1-e^2)/e atanh e)
            e = math.sqrt(1 - c * c / (a * a))
            exact = 2 * np.pi * a * a * (1 + (1 - e * e) / e * math.atanh(e))
        assert oracle.ellipsoid_area([a, a, c]) == pytest.approx(exact, rel=0.011)


@pytest.mark.parametrize("K", [2, 3, 5])
def test_merge_identical_children(K):
    """Identical children: the parent equals the child (mean, covariance, SH) and its falloff is
    K times the child's opacity, since sum(w'_i) / S_p = K o S / S (Sec. 4.1, falloff)."""
    rng = np.random.default_rng(K)
    r = _random_row(rng)
    p = oracle.merge_rows(np.stack([r] * K))
    np.testing.assert_allclose(p[:3], r[:3], atol=1e-14)
    np.testing.assert_allclose(_cov(p[3:6], p[6:10]), _cov(r[3:6], r[6:10]), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(p[11:], r[11:], atol=1e-14)
    assert p[10] == pytest.approx(K * r[10], rel=1e-10)


def test_merge_moments_match_monte_carlo_mixture():
    """Eq. merge is moment matching of the weighted mixture.  Children share one scale triplet
    (so S_i is equal and w_i = o_i / sum o); the merged mean/covariance must match the sample
    moments of 4M draws from that mixture."""
    rng = np.random.default_rng(11)
    s = np.array([0.3, 0.1, 0.05])
    rows = [_random_row(rng, scale=s) for _ in range(3)]
    rows[0][10], rows[1][10], rows[2][10] = 0.9, 0.3, 0.5
    p = oracle.merge_rows(np.stack(rows))
    w = np.array([r[10] for r in rows])
    w /= w.sum()
    n = 4_000_000
    comp = rng.choice(3, size=n, p=w)
    pts = np.empty((n, 3))
    for i, r in enumerate(rows):
        k = comp == i
        L = np.linalg.cholesky(_cov(r[3:6], r[6:10]))
        pts[k] = r[:3] + rng.standard_normal((k.sum(), 3)) @ L.T
    mu_s, cov_s = pts.mean(0), np.cov(pts.T)
    np.testing.assert_allclose(p[:3], mu_s, atol=3e-3)
    np.testing.assert_allclose(_cov(p[3:6], p[6:10]), cov_s, atol=4e-3 * np.abs(cov_s).max())
    # SH uses the same weights: recover w from the merged mean (mean is pinned above)
    np.testing.assert_allclose(p[11:], sum(wi * r[11:] for wi, r in zip(w, rows)), atol=1e-12)


def test_merge_weights_follow_surface_area():
    """Two children, equal opacity, different size, same centre: the heavier weight goes to the
    larger surface (w'_i = o_i S_i, Sec. 4.1): merged SH lands at S-weighted average."""
    small = _row([0, 0, 0], [0.1, 0.1, 0.1], [1, 0, 0, 0], 0.5, np.full(48, 0.0))
    big = _row([0, 0, 0], [0.3, 0.3, 0.3], [1, 0, 0, 0], 0.5, np.full(48, 1.0))
    p = oracle.merge_rows(np.stack([small, big]))
    # spheres: S = 4 pi r^2 exactly, so w_big = 0.09 / (0.09 + 0.01)
    np.testing.assert_allclose(p[11:], 0.9, atol=1e-12)
    # parent covariance = weighted covariances (same means) -> isotropic (0.1*0.01+0.9*0.09)
    np.testing.assert_allclose(_cov(p[3:6], p[6:10]), np.eye(3) * (0.1 * 0.01 + 0.9 * 0.09), atol=1e-12)
    # falloff = (0.5*S_s + 0.5*S_b) / S_p with every S a sphere area
    rp2 = 0.1 * 0.01 + 0.9 * 0.09
    assert p[10] == pytest.approx(0.5 * (0.01 + 0.09) / rp2, rel=1e-10)


# ------------------------------------------------------------------ orientation matching (Sec. 4.2)

def _proper_signed_perms():
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            P = np.zeros((3, 3))
            for j in range(3):
                P[perm[j], j] = signs[j]
            if np.linalg.det(P) > 0:
                out.append(P)
    return out


def test_orientation_matching_minimises_rotation_and_keeps_covariance():
    rng = np.random.default_rng(5)
    perms = _proper_signed_perms()
    assert len(perms) == 24
    for _ in range(40):
        par, ch = _random_row(rng), _random_row(rng)
        m = oracle.match_orientation(par, ch)
        np.testing.assert_allclose(_cov(m[3:6], m[6:10]), _cov(ch[3:6], ch[6:10]), rtol=1e-10, atol=1e-14)
        Rp, Rc = _rotmat(par[6:10]), _rotmat(ch[6:10])
        ang = [np.arccos(np.clip((np.trace(Rp.T @ Rc @ P) - 1) / 2, -1, 1)) for P in perms]
        got = oracle.rotation_angle(par[6:10], m[6:10])
        assert got <= min(ang) + 1e-9
        assert np.dot(m[6:10], par[6:10]) >= 0


# ------------------------------------------------------------------ BVH (Sec. 4.1)

def test_bvh_structure_and_boxes():
    sc, h = scenes.tiny()
    L = sc.leaves.n
    N = h.n
    assert N == 2 * L - 1
    assert h.parent[0] == -1
    # BFS numbering: parent < child, children contiguous, every non-root has one parent
    for v in range(N):
        cs, cc = h.child_start[v], h.child_count[v]
        assert cc in (0, 2)
        for c in range(cs, cs + cc):
            assert h.parent[c] == v and c > v
    # each leaf appears exactly once (a leaf's Gaussian covariance equals one input leaf's)
    leaves = np.flatnonzero(h.child_count == 0)
    assert len(leaves) == L
    key_in = {tuple(np.round(m, 6)) for m in sc.leaves.mean}
    assert {tuple(np.round(h.mean[v], 6)) for v in leaves} == key_in
    # boxes nest
    for v in range(1, N):
        p = h.parent[v]
        assert np.all(h.box_min[p] <= h.box_min[v]) and np.all(h.box_max[p] >= h.box_max[v])
    # leaf box = tight AABB of the 3-sigma ellipsoid (sampled surface points touch every face)
    rng = np.random.default_rng(0)
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    for v in leaves[:50]:
        R = _rotmat(h.rot[v])
        pts = h.mean[v] + 3.0 * (u * h.scale[v]) @ R.T
        ext = np.maximum(pts.max(0) - h.mean[v], h.mean[v] - pts.min(0))
        half = 0.5 * (h.box_max[v] - h.box_min[v])
        assert np.all(pts.max(0) <= h.box_max[v] + 1e-5) and np.all(pts.min(0) >= h.box_min[v] - 1e-5)
        np.testing.assert_allclose(ext, half, rtol=2e-2)


def test_bvh_median_split_on_longest_axis():
    sc, h = scenes.tiny()
    N = h.n
    # leaves under each node
    under = [None] * N
    for v in range(N - 1, -1, -1):
        if h.child_count[v] == 0:
            under[v] = [v]
        else:
            under[v] = under[h.child_start[v]] + under[h.child_start[v] + 1]
    for v in range(N):
        if h.child_count[v] == 0:
            continue
        ext = h.box_max[v].astype(np.float64) - h.box_min[v].astype(np.float64)
        axis = int(np.argmax(ext))
        left, right = under[h.child_start[v]], under[h.child_start[v] + 1]
        assert len(left) == len(under[v]) // 2
        assert h.mean[left, axis].max() <= h.mean[right, axis].min()


# ------------------------------------------------------------------ cut (Sec. 4.2)

def _paths_hit_once(h, cut):
    inc = np.zeros(h.n, bool)
    inc[cut] = True
    for leaf in np.flatnonzero(h.child_count == 0):
        v, hits = leaf, 0
        while v >= 0:
            hits += inc[v]
            v = h.parent[v]
        if hits != 1:
            return False
    return True


def test_cut_special_cases_and_invariants():
    sc, h = scenes.tiny()
    cam = sc.cameras[0]
    ids, t = oracle.select_cut(synth.with_tau(cam, 0.0), h)
    np.testing.assert_array_equal(ids, np.flatnonzero(h.child_count == 0))   # tau = 0: the leaves
    assert np.all(t == 0)
    ids, t = oracle.select_cut(synth.with_tau(cam, float("inf")), h)
    np.testing.assert_array_equal(ids, [0])                                   # tau = inf: the root
    eps = oracle.granularity(cam, h)
    assert np.all(eps[1:] <= eps[h.parent[1:]])                               # parent never smaller
    for tau in [0.5, 2, 6, 20, 100, 1000]:
        c = synth.with_tau(cam, tau)
        ids, t = oracle.select_cut(c, h)
        assert np.all(np.diff(ids) > 0)
        np.testing.assert_array_equal(ids, oracle.select_cut_descent(c, h))
        assert _paths_hit_once(h, ids)
        assert np.all((t >= 0) & (t <= 1))
        inner = (eps[ids] < tau) & (h.parent[ids] >= 0)
        assert np.all(t[~inner] == 0)




@pytest.mark.parametrize("seed", range(12))
def test_cut_invariants_on_random_trees_and_cameras(seed):
    """The cut (Sec. 4.2) on seeded random trees of 1 to 300 leaves, seen from random positions
    (outside and inside the leaves' cube, any direction) at random tau, including 0 and infinity:
    ids ascending, equal to the recursive descent from the root, every root-to-leaf path meets the
    cut once, weights in [0, 1].  At tau = 0 the cut is the leaves; at tau = infinity it is the root
    when the camera is outside the root's box, and otherwise the nodes of finite granularity
    closest to the root (a box holding the camera is at distance 0: infinitely coarse)."""
    rng = np.random.default_rng([seed, 77])
    n_leaves = int(rng.choice([1, 2, 3, 17, 64, 300]))
    sc = synth.tiny_scene(seed=100 + seed, n_leaves=n_leaves)
    h = oracle.build_tree(sc.leaves)
    assert h.n == 2 * n_leaves - 1
    for k in range(4):
        pos = rng.uniform(-15.0, 25.0, 3) if k % 2 else rng.uniform(2.0, 8.0, 3)
        fwd = rng.normal(size=3)
        up = np.cross(fwd, rng.normal(size=3))
        for tau in (0.0, float(np.exp(rng.uniform(np.log(0.1), np.log(500.0)))), float("inf")):
            cam = synth.look_camera(pos, fwd, up, 160, 120, float(rng.uniform(30, 100)), tau)
            ids, t = oracle.select_cut(cam, h)
            assert np.all(np.diff(ids) > 0)
            np.testing.assert_array_equal(ids, oracle.select_cut_descent(cam, h))
            assert _paths_hit_once(h, ids)
            assert np.all((t >= 0) & (t <= 1))
            if tau == 0.0:
                np.testing.assert_array_equal(ids, np.flatnonzero(h.child_count == 0))
            if tau == float("inf"):
                inside = np.all(pos >= h.box_min[0]) and np.all(pos <= h.box_max[0])
                if not inside:
                    np.testing.assert_array_equal(ids, [0])
                    assert t[0] == 0
                else:
                    eps = oracle.granularity(cam, h)
                    cut_leaf = h.child_count[ids] == 0
                    assert np.all(np.isfinite(eps[ids]) | cut_leaf)
                    assert not np.isfinite(eps[0]) and 0 not in ids

@pytest.mark.parametrize("tau", [3.0, 15.0])
def test_cut_rule_is_local_under_a_joined_root(tau):
    """The cut rule is local (Sec. 4.2: a node is in the cut iff its granularity is below tau and its
    parent's is not, or it is a leaf under an expanded parent), so joining two copies of a tree
    under a new root that is expanded leaves each copy's cut and weights as the copy's own (the test
    tree of the several-wave scan, here at 100k leaves).  The joined tree is checked for a valid
    hierarchy first: every node but the root is one child of its parent, parents come before their
    children, and child boxes nest in their parent's."""
    sc, h1 = scenes.corridor(100_000)
    h = scenes.two_corridors(100_000)
    n1 = h1.n
    assert h.n == 2 * n1 + 1
    par, cs, cc = h.parent, h.child_start, h.child_count
    assert par[0] == -1 and np.all(par[1:] < np.arange(1, h.n))
    inner = np.flatnonzero(cc > 0)
    kids = np.concatenate([cs[inner] + k for k in range(2)])
    assert np.all(cc[inner] == 2)
    np.testing.assert_array_equal(np.sort(kids), np.arange(1, h.n))   # each non-root node once
    assert np.all(par[kids] == np.concatenate([inner, inner]))
    assert np.all(h.box_min[1:] >= h.box_min[par[1:]]) and np.all(h.box_max[1:] <= h.box_max[par[1:]])
    cam = synth.with_tau(sc.cameras[0], tau)
    ids, t = oracle.select_cut(cam, h)
    o1, t1 = oracle.select_cut(cam, h1)
    assert 0 not in ids and 1 not in ids      # the new root and the first copy's root are expanded
    first = (ids >= 3) & (ids < n1 + 2)       # the first copy's nodes other than its root: id - 2
    np.testing.assert_array_equal(ids[first] - 2, o1)
    np.testing.assert_array_equal(t[first].view(np.uint32), t1.view(np.uint32))
    second = ids >= n1 + 2                    # the second copy, shifted down the street
    assert second.sum() > 0 and first.sum() + second.sum() == len(ids)

def test_granularity_is_projected_box_size():
    """eps(n) = f * (largest box side) / (distance to the box); check against a direct fp64
    evaluation of the worst-case projected size of a box edge seen head-on."""
    lv = scenes.leaves_from([[0, 0, 10]], [[0.2, 0.1, 0.05]], [[1, 0, 0, 0]], [0.5])
    h = oracle.build_tree(lv)
    cam = scenes.axis_camera(64, 64, f=100.0)
    eps = oracle.granularity(cam, h)[0]
    # box: +-0.6 in x, +-0.3 in y, +-0.15 in z; nearest point at z = 9.85 on the axis
    assert eps == pytest.approx(100.0 * 1.2 / 9.85, rel=1e-6)


# ------------------------------------------------------------------ projection / footprint (Sec. 3.1, Eq. blend)

def _single(mu, s, q, o, dc=0.3):
    sh = np.zeros(48)
    sh[0:3] = dc
    h = oracle.build_tree(scenes.leaves_from([mu], [s], [q], [o], sh))
    return h


def test_isotropic_footprint_closed_form():
    """One isotropic Gaussian on the optical axis: Sigma' = (f sigma / z)^2 I, the filtered
    Sigma'_f adds 0.3 I, the peak pixel is o comp c, and the image integrates to
    o comp c sqrt((2 pi)^2 |Sigma'_f|) (the paper's integral of G, Sec. 4.1)."""
    f32 = lambda x: float(np.float32(x))      # inputs are stored in fp32
    f, sig, z, o, lp, dc = 200.0, f32(0.05), 5.0, f32(0.8), f32(0.3), f32(0.3)
    h = _single([0, 0, z], [sig] * 3, [1, 0, 0, 0], o, dc)
    cam = scenes.axis_camera(256, 256, f, cx=128.5, cy=128.5, tau=6.0)
    opts = oracle.Opts(alpha_floor=0.0, t_min=0.0)
    fr = oracle.render(cam, h, opts)
    v = fr.val64[0]
    s2 = (f * sig / z) ** 2
    det_f = (s2 + lp) ** 2
    np.testing.assert_allclose([v[2], v[3], v[4]], [1 / (s2 + lp), 0.0, 1 / (s2 + lp)], rtol=1e-12, atol=1e-15)
    comp = s2 / (s2 + lp)
    assert v[5] == pytest.approx(o * comp, rel=1e-12)
    c = 0.5 + dc * 0.5 / math.sqrt(math.pi)
    assert fr.image[0, 128, 128] == pytest.approx(o * comp * c, rel=1e-12)
    total = fr.image[0].sum()
    assert total == pytest.approx(o * comp * c * 2 * np.pi * math.sqrt(det_f), rel=1e-9)


def test_anisotropic_projection_matches_numeric_jacobian():
    """EWA: Sigma' = J W Sigma W^T J^T with J the Jacobian of the pinhole map at the mean; J is
    taken here by central differences of u(x) = f x/z + c (no clamp active)."""
    rng = np.random.default_rng(2)
    for _ in range(5):
        mu = np.array([rng.uniform(-1, 1), rng.uniform(-0.5, 0.5), rng.uniform(4, 8)])
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        s = np.exp(rng.normal(-2.5, 0.5, 3))
        h = _single(mu, s, q, 0.6)
        ang = rng.normal(size=3) * 0.1
        R = Rotation.from_rotvec(ang).as_matrix().astype(np.float32)
        T = rng.normal(size=3).astype(np.float32) * 0.1
        cam = synth.Camera(R, T, 300.0, 310.0, 160.0, 120.0, 320, 240, 6.0)
        fr = oracle.render(cam, h)
        v = fr.val64[0]
        Rd, Td = R.astype(np.float64), T.astype(np.float64)
        mu_f = h.mean[0].astype(np.float64)

        def proj(x):
            xc = Rd @ x + Td
            return np.array([cam.fx * xc[0] / xc[2] + cam.cx, cam.fy * xc[1] / xc[2] + cam.cy])
        J = np.stack([(proj(mu_f + e) - proj(mu_f - e)) / 2e-6 for e in np.eye(3) * 1e-6], axis=1)
        Sig = _cov(h.scale[0].astype(np.float64), h.rot[0].astype(np.float64))
        S2 = J @ Sig @ J.T + float(np.float32(0.3)) * np.eye(2)
        conic = np.array([[v[2], v[3]], [v[3], v[4]]])
        np.testing.assert_allclose(np.linalg.inv(conic), S2, rtol=1e-6)
        np.testing.assert_allclose(v[:2], proj(mu_f), rtol=1e-12)


# ------------------------------------------------------------------ transition (Sec. 4.2, Eq. alphap, t_interp)

def test_transition_is_continuous_at_both_ends():
    """At tau = eps(p) the two children enter with t = 1: they take the parent's attributes
    and blend with alpha' each, reproducing the parent exactly (Eq. alphap).  Just above
    eps(n) (t -> 0) they render as themselves."""
    lv = scenes.leaves_from([[-0.05, 0.0, 6.0], [0.06, 0.02, 6.1]], [[0.05, 0.03, 0.04], [0.04, 0.05, 0.03]],
                            [[1, 0, 0, 0], [0.9, 0.1, 0.3, 0.2]], [0.7, 0.8],
                            np.random.default_rng(3).normal(0, 0.3, (2, 48)))
    h = oracle.build_tree(lv)
    cam = scenes.axis_camera(96, 96, 300.0)
    eps = oracle.granularity(cam, h)
    assert eps[0] > eps[1] and eps[0] > eps[2]
    par = oracle.render(synth.with_tau(cam, float(np.nextafter(np.float32(eps[0]), np.float32(np.inf)))), h)
    assert list(par.ids) == [0]
    kids = oracle.render(synth.with_tau(cam, float(eps[0])), h)
    assert list(kids.ids) == [1, 2] and np.all(kids.t == 1.0)
    # children at t=1 draw the parent's footprint with alpha' each; equal wherever alpha' stays above
    # the 1/255 floor (the floor is applied per splat, so the outer rim may differ)
    inner = par.image[0] > 0.05 * par.image[0].max()
    np.testing.assert_allclose(kids.image[:, inner], par.image[:, inner], rtol=1e-12, atol=1e-14)
    # near the lower end (t -> 0) the children render as themselves: mirror-symmetric children
    # share one granularity, so both reach t ~ 0 together
    sh = np.random.default_rng(4).normal(0, 0.3, (2, 48))
    lv = scenes.leaves_from([[-0.12, 0.0, 6.0], [0.12, 0.0, 6.0]], [[0.05, 0.03, 0.04]] * 2,
                            [[1, 0, 0, 0]] * 2, [0.7, 0.8], sh)
    h = oracle.build_tree(lv)
    eps = oracle.granularity(cam, h)
    assert eps[1] == eps[2] < eps[0]
    lo = float(np.nextafter(np.float32(eps[1]), np.float32(np.inf)))
    a = oracle.render(synth.with_tau(cam, lo), h)
    b = oracle.render(synth.with_tau(cam, lo), h, oracle.Opts(interpolate=0))
    assert list(a.ids) == [1, 2] and np.all(a.t < 1e-5)
    np.testing.assert_allclose(a.image, b.image, atol=1e-5)


def test_alpha_prime_recovers_parent_opacity():
    """At t = 1 the K = 2 children blend to transmittance (1 - alpha')^2 = 1 - alpha_p (Eq. alphap):
    two small children offset so the parent's box is larger (a transition window exists)."""
    lv = scenes.leaves_from([[-0.01, 0, 5.0], [0.01, 0, 5.0]], [[0.05] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.3, 0.3])
    h = oracle.build_tree(lv)
    cam = scenes.axis_camera(64, 64, 200.0, cx=32.5, cy=32.5)
    eps = oracle.granularity(cam, h)
    assert eps[0] > eps[1] and eps[0] > eps[2]
    fr = oracle.render(synth.with_tau(cam, float(eps[0])), h, oracle.Opts(alpha_floor=0.0, t_min=0.0))
    assert list(fr.ids) == [1, 2] and np.all(fr.t == 1.0)
    v = fr.val64[0]
    dx, dy = 32.5 - v[0], 32.5 - v[1]
    G = math.exp(-0.5 * (v[2] * dx * dx + 2 * v[3] * dx * dy + v[4] * dy * dy))
    ap = min(float(np.float32(0.99)), v[6] * G)
    assert 0.3 < ap < 0.9
    assert fr.T_final[32, 32] == pytest.approx(1 - ap, rel=1e-12)


# ------------------------------------------------------------------ blending rules

def test_tiled_equals_bruteforce_over_tile_shapes():
    lv, cam = scenes.small_random_scene(n_leaves=96, res=(70, 45))
    h = oracle.build_tree(lv)
    for tw, th in [(16, 16), (8, 8), (32, 8), (8, 32)]:
        opts = oracle.Opts(tile_w=tw, tile_h=th)
        fr = oracle.render(cam, h, opts)
        bf = oracle.blend_bruteforce(cam, fr, opts)
        np.testing.assert_allclose(fr.image, bf, atol=1e-13)
        assert fr.image.max() > 0.1



@pytest.mark.parametrize("seed", range(8))
def test_tiled_equals_bruteforce_on_random_scenes(seed):
    """The tiled blend (depth sort, tile lists, per-tile front-to-back walk) equals the per-pixel
    brute force over every splat on seeded random scenes at several tau (so that interpolated
    splats, t != 0, take part) and a random tile shape."""
    rng = np.random.default_rng([seed, 55])
    lv, cam = scenes.small_random_scene(n_leaves=int(rng.integers(8, 120)), seed=1000 + seed, res=(61, 37),
                                        log_scale=float(rng.uniform(-3.0, -2.0)))
    h = oracle.build_tree(lv)
    tw, th = [(16, 16), (8, 8), (32, 8), (8, 32)][int(rng.integers(4))]
    opts = oracle.Opts(tile_w=tw, tile_h=th)
    n_interp = 0
    for tau in (0.0, 2.0, 6.0, 20.0):
        fr = oracle.render(synth.with_tau(cam, tau), h, opts)
        bf = oracle.blend_bruteforce(synth.with_tau(cam, tau), fr, opts)
        np.testing.assert_allclose(fr.image, bf, atol=1e-13)
        n_interp += int(np.sum(fr.t != 0))
    assert n_interp > 0

def test_alpha_floor_and_transmittance_stop():
    """A splat whose alpha never reaches 1/255 changes nothing; the transmittance stop halts
    BEFORE the splat that would take T below 1e-4, so nothing behind it is added."""
    cam = scenes.axis_camera(32, 32, 100.0, cx=16.5, cy=16.5)
    off = -0.5 * 2 * math.sqrt(math.pi)          # DC coefficient that zeroes a channel
    sh_red = np.zeros(48); sh_red[0:3] = [1.0, off, off]
    sh_blue = np.zeros(48); sh_blue[0:3] = [off, off, 1.0]
    base = ([[0, 0, 5.0]], [[0.2] * 3], [[1, 0, 0, 0]], [0.5], sh_red[None])
    faint = ([[0, 0, 4.0]], [[0.2] * 3], [[1, 0, 0, 0]], [0.003], sh_blue[None])
    h1 = oracle.build_tree(scenes.leaves_from(*base))
    img1 = oracle.render(synth.with_tau(cam, 0.0), h1).image
    lv2 = scenes.leaves_from(*[np.concatenate([a, b]) for a, b in zip(base, faint)])
    img2 = oracle.render(synth.with_tau(cam, 0.0), oracle.build_tree(lv2)).image
    np.testing.assert_array_equal(img1, img2)
    # four opaque layers with alpha clamped at 0.95: T 1 -> .05 -> .0025 -> 1.25e-4 -> (6e-6: stop)
    means = [[0, 0, 4.0], [0, 0, 4.5], [0, 0, 5.0], [0, 0, 5.5]]
    sh = np.stack([sh_red, sh_red, sh_red, sh_blue])
    lv3 = scenes.leaves_from(means, [[0.3] * 3] * 4, [[1, 0, 0, 0]] * 4, [50.0] * 4, sh)
    fr = oracle.render(synth.with_tau(cam, 0.0), oracle.build_tree(lv3), oracle.Opts(alpha_clamp=0.95))
    assert fr.image[2, 16, 16] == 0.0
    assert fr.image[0, 16, 16] > 0.5
    assert fr.T_final[16, 16] == pytest.approx((1 - float(np.float32(0.95))) ** 3, rel=1e-9)
    assert fr.n_contrib[16, 16] == 3


# ------------------------------------------------------------------ adjoint (Sec. 5.1, Sec. 7.1, Sec. 7.3)

def _fd_scene(seed=9):
    lv, cam = scenes.small_random_scene(n_leaves=40, res=(40, 32), seed=seed, log_scale=-2.2)
    h = oracle.build_tree(lv)
    eps = oracle.granularity(cam, h)
    best = None
    for tau in np.quantile(eps[h.child_count > 0], np.linspace(0.05, 0.95, 19)):
        ids, t = oracle.select_cut(synth.with_tau(cam, float(tau)), h)
        k = int(np.sum((t > 0.05) & (t < 0.95)))
        if best is None or k > best[0]:
            best = (k, float(tau))
    assert best[0] >= 4
    return h, synth.with_tau(cam, best[1])


@pytest.mark.parametrize("seed", [9, 21, 33])
def test_backward_matches_finite_differences(seed):
    """The analytic adjoint (interpolation -> projection -> SH -> blend, with the manual alpha'
    derivative) against central differences of the fp64 track with the decisions held fixed, on
    three seeded scenes.  Parameters whose one-sided differences disagree by more than 10% sit on a
    kink (a clamp) and are skipped."""
    h, cam = _fd_scene(seed)
    opts = oracle.Opts()
    a64 = oracle.Attrs64.of(h)
    fr = oracle.render(cam, h, opts, a64)
    rng = np.random.default_rng(1)
    w = rng.normal(size=fr.image.shape)
    g = oracle.backward(cam, h, fr, w, opts, a64)
    touched = np.unique(np.concatenate([fr.ids, h.parent[fr.ids][h.parent[fr.ids] >= 0]]))
    fields = [("mean", 3), ("scale", 3), ("rot", 4), ("opacity", 1), ("sh", 48)]
    col = 0
    spans = []
    for name, k in fields:
        spans.append((name, col, k))
        col += k
    checked = skipped = 0
    gmax = np.abs(g).max()
    for node in rng.choice(touched, size=min(len(touched), 30), replace=False):
        for name, c0, k in spans:
            for j in (range(k) if k <= 4 else rng.choice(k, 6, replace=False)):
                arr = getattr(a64, name)
                flat = arr.reshape(arr.shape[0], -1)
                theta = flat[node, j]
                step = 1e-6 * max(abs(theta), 0.05)
                vals = []
                for d in (step, -step):
                    flat[node, j] = theta + d
                    vals.append(oracle.weighted_image_sum(cam, h, fr, w, opts, a64))
                flat[node, j] = theta
                f0 = oracle.weighted_image_sum(cam, h, fr, w, opts, a64)
                fwd, bwd = (vals[0] - f0) / step, (f0 - vals[1]) / step
                if abs(fwd - bwd) > 0.1 * max(abs(fwd), abs(bwd), 1e-6 * gmax):
                    skipped += 1
                    continue
                fd = (vals[0] - vals[1]) / (2 * step)
                an = g[node, c0 + j]
                assert abs(fd - an) <= 1e-4 * max(abs(fd), abs(an)) + 1e-7 * gmax, (name, node, j, fd, an)
                checked += 1
    assert checked > 300 and skipped < 0.1 * checked


def test_backward_freeze_leaves_and_parent_share():
    """Frozen leaves receive nothing (Sec. 7.1); a cut node with 0 < t < 1 sends gradient to its
    parent, in proportion t : (1 - t) for the linearly interpolated SH coefficients."""
    h, cam = _fd_scene()
    opts = oracle.Opts()
    fr = oracle.render(cam, h, opts)
    w = np.random.default_rng(2).normal(size=fr.image.shape)
    g = oracle.backward(cam, h, fr, w, opts)
    gf = oracle.backward(cam, h, fr, w, opts, freeze_leaves=1)
    leaf = h.child_count == 0
    assert np.all(gf[leaf] == 0)
    np.testing.assert_allclose(gf[~leaf], g[~leaf], rtol=1e-12, atol=1e-15)
    # a leaf child whose sibling subtree is not in the cut: only this child feeds the parent's SH
    for i, (n, t) in enumerate(zip(fr.ids, fr.t)):
        p = h.parent[n]
        if not (0.05 < t < 0.95) or not leaf[n]:
            continue
        sib = h.child_start[p] + (1 - (n - h.child_start[p]))
        if sib in set(fr.ids.tolist()) or not leaf[sib]:
            continue
        np.testing.assert_allclose(g[p, 11:] * (1 - t), g[n, 11:] * t, rtol=1e-9, atol=1e-15)


# ------------------------------------------------------------------ fp32 decision track (Sec. 3.1 Eq. alpha, Eq. alphap)
#
# The oracle takes every integer decision (tile rectangle, alpha floor, transmittance stop) in an
# fp32 track (project_f / alpha_f: the conic pre-scaled to a base-2 exponent, fp32 arithmetic in a
# fixed order) and every value in an fp64 track (project_d / alpha_d), which the tests above pin
# by closed forms, a numeric Jacobian and finite differences.  The pins below tie the fp32 track
# to the fp64 track at every (pixel, splat) pair of seeded scenes, binary and K-ary (K = 2, 3, 5)
# transitions included, so that a dropped term, a wrong sign or a wrong base-2 factor in the
# decision track fails them.

_KH = float(np.float32(-0.72134752044448170))     # the decision track's -log2(e)/2
_KL = float(np.float32(1.44269504088896341))      # and log2(e)


def _box3(mean, scale, q):
    R = _rotmat(q)
    he = 3 * np.sqrt(((R * np.asarray(scale, np.float64)[None, :]) ** 2).sum(1))
    return mean - he, mean + he


def _kary_hierarchy(K, rng, depth=3.0):
    """A root merged (Eq. merge) from K leaf children, leaf boxes the 3-sigma AABBs, the root box
    their union: one K-child transition (Eq. alphap with K children, Sec. 5.2)."""
    mean = np.c_[rng.uniform(-0.15, 0.15, K), rng.uniform(-0.15, 0.15, K), depth + rng.uniform(-0.1, 0.1, K)]
    scale = np.exp(rng.normal(-3.0, 0.3, (K, 3)))
    q = rng.normal(size=(K, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    rows = np.c_[mean, scale, q, rng.uniform(0.3, 0.95, K), rng.normal(0, 0.3, (K, 48))]
    allr = np.vstack([oracle.merge_rows(rows)[None], rows]).astype(np.float32)
    bmin = np.empty((K + 1, 3), np.float32)
    bmax = np.empty((K + 1, 3), np.float32)
    for i in range(K):
        bmin[i + 1], bmax[i + 1] = _box3(mean[i], scale[i], q[i])
    bmin[0], bmax[0] = bmin[1:].min(0), bmax[1:].max(0)
    c = np.ascontiguousarray
    return oracle.Hierarchy(c(allr[:, 0:3]), c(allr[:, 3:6]), c(allr[:, 6:10]), c(allr[:, 10]), c(allr[:, 11:59]),
                            bmin, bmax, np.r_[-1, np.zeros(K)].astype(np.int32),
                            np.r_[1, np.zeros(K)].astype(np.int32), np.r_[K, np.zeros(K)].astype(np.int32))


def _decision_track_frames():
    """Rendered frames of a 200-leaf binary scene at five tau and of K-child transitions at four tau
    each, every one with splats at 0 < t < 1."""
    opts = oracle.Opts()
    lv, cam = scenes.small_random_scene(n_leaves=200, res=(96, 80), seed=11)
    h = oracle.build_tree(lv)
    eps = oracle.granularity(cam, h)
    out = []
    for tau in np.quantile(eps[h.child_count > 0], [0.1, 0.3, 0.5, 0.7, 0.9]):
        c = synth.with_tau(cam, float(tau))
        out.append((c, oracle.render(c, h, opts)))
    rng = np.random.default_rng(5)
    kcam = scenes.axis_camera(64, 64, 120.0)
    for K in (2, 3, 5):
        for _ in range(2):
            hk = _kary_hierarchy(K, rng)
            ek = oracle.granularity(kcam, hk)
            assert ek[0] > ek[1:].max()
            for tau in np.linspace(ek[1:].max(), ek[0], 6)[1:-1]:
                c = synth.with_tau(kcam, float(tau))
                fr = oracle.render(c, hk, opts)
                assert list(fr.ids) == list(range(1, K + 1)) and np.all((fr.t > 0) & (fr.t < 1))
                out.append((c, fr))
    return opts, out


def test_decision_track_records_match_value_track():
    """Per visible splat: the base-2 pre-scaled conic (ca, cb, cc) of the decision record is
    (-A/2, -B, -C/2) log2(e) of the value track's conic; centre, opacities, t, K and depth agree."""
    _, frames = _decision_track_frames()
    n_t = 0
    for _, fr in frames:
        vis = fr.rect[:, 0] >= 0
        r, v = fr.rec32[vis].astype(np.float64), fr.val64[vis]
        A, B, Cc = r[:, 2] / _KH, -r[:, 3] / _KL, r[:, 4] / _KH
        scale = np.sqrt(v[:, 2] * v[:, 4])
        assert np.all(v[:, 2] > 0) and np.all(v[:, 4] > 0)
        np.testing.assert_array_less(np.abs(A - v[:, 2]), 1e-5 * v[:, 2])
        np.testing.assert_array_less(np.abs(Cc - v[:, 4]), 1e-5 * v[:, 4])
        np.testing.assert_array_less(np.abs(B - v[:, 3]), 1e-5 * scale)
        np.testing.assert_array_less(np.abs(r[:, 0:2] - v[:, 0:2]), 1e-3)                 # pixels
        np.testing.assert_array_less(np.abs(r[:, 5:7] - v[:, 5:7]), 1e-5 * np.abs(v[:, 5:7]) + 1e-30)
        np.testing.assert_array_equal(r[:, 7], v[:, 7])                                     # t
        np.testing.assert_array_equal(r[:, 8], v[:, 8])                                     # K
        np.testing.assert_array_less(np.abs(r[:, 9] - v[:, 12]), 1e-6 * v[:, 12])          # depth
        n_t += int(np.sum(r[:, 7] > 0))
    assert n_t > 300


def _rect_pairs(cam, fr, opts):
    S, PX, PY = [], [], []
    for i in np.nonzero(fr.rect[:, 0] >= 0)[0]:
        x0, x1, y0, y1 = fr.rect[i]
        xs = np.arange(x0 * opts.tile_w, min((x1 + 1) * opts.tile_w, cam.width))
        ys = np.arange(y0 * opts.tile_h, min((y1 + 1) * opts.tile_h, cam.height))
        X, Y = np.meshgrid(xs, ys)
        S.append(np.full(X.size, i))
        PX.append(X.ravel() + 0.5)
        PY.append(Y.ravel() + 0.5)
    return np.concatenate(S), np.concatenate(PX), np.concatenate(PY)


@functools.lru_cache(maxsize=None)
def _street_frames():
    """Two 320x180 views of a 100k-leaf street corridor: kilometre-scale world coordinates, metre-scale
    camera-space ones (the large-scene setting of Sec. 6)."""
    opts = oracle.Opts()
    sc = synth.corridor_scene(seed=3, n_leaves=100_000)
    h = oracle.build_tree(sc.leaves)
    _, views = synth.optimisation_views(seed=3, width=320, height=180)
    return opts, [(views[k], oracle.render(views[k], h, opts)) for k in (0, 5)]


def _ulp(x):
    return np.spacing(np.abs(np.asarray(x, np.float64)).astype(np.float32)).astype(np.float64)


def _uv_resolution_bound(cam, fr, S, PX, PY):
    """Relative alpha error that the fp32 representation of the splat's screen position alone allows:
    |dp/du| du + |dp/dv| dv with p the natural exponent of the value track and du, dv four units in
    the last place of fp32 screen coordinates (u = fx x/z + cx is resolved at the scale of the
    image, max(|u|, width)), plus 2e-6 (1 + |p|) for the rounding of the exponent itself."""
    v = fr.val64[S]
    dx, dy = PX - v[:, 0], PY - v[:, 1]
    A, B, Cc = v[:, 2], v[:, 3], v[:, 4]
    p = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
    du = 4 * _ulp(np.maximum(np.abs(v[:, 0]), cam.width))
    dv = 4 * _ulp(np.maximum(np.abs(v[:, 1]), cam.height))
    return np.abs(A * dx + B * dy) * du + np.abs(B * dx + Cc * dy) * dv + 2e-6 * (1 + np.abs(p))


def test_decision_track_keeps_metre_precision_in_kilometre_scenes():
    """On a street corridor 1 km long the decision track's splat centres stay within a few fp32 units
    in the last place of the exact ones (the world -> camera transform must not cancel the
    kilometre-scale coordinates away), and its alpha matches the value track's alpha within the
    resolution of fp32 screen coordinates at every pair with alpha >= 1e-3."""
    opts, frames = _street_frames()
    n_pairs = 0
    for cam, fr in frames:
        vis = fr.rect[:, 0] >= 0
        r, v = fr.rec32[vis].astype(np.float64), fr.val64[vis]
        np.testing.assert_array_less(np.abs(r[:, 0] - v[:, 0]), 4 * _ulp(np.maximum(np.abs(v[:, 0]), cam.width)))
        np.testing.assert_array_less(np.abs(r[:, 1] - v[:, 1]), 4 * _ulp(np.maximum(np.abs(v[:, 1]), cam.height)))
        np.testing.assert_array_less(np.abs(r[:, 9] - v[:, 12]), 4e-7 * v[:, 12])         # depth
        assert np.sum(r[:, 7] > 0) > 5000
        S, PX, PY = _rect_pairs(cam, fr, opts)
        a32, a64 = oracle.pair_alpha(fr, S, PX, PY, opts)
        m = a64 >= 1e-3
        bound = _uv_resolution_bound(cam, fr, S, PX, PY)
        np.testing.assert_array_less(np.abs(a32.astype(np.float64) - a64)[m], (bound * a64)[m])
        n_pairs += int(m.sum())
    assert n_pairs > 500_000


def test_decision_alpha_matches_value_alpha():
    """At every pixel of every splat's tile rectangle the fp32 alpha the decisions use equals the
    fp64 alpha = (1-t) min(0.99, o_n G) + t (1 - (1 - min(0.99, o_p G))^(1/K)) within 1e-5 relative
    wherever alpha >= 1e-3 (the oracle's ambiguity band around the 1/255 floor is 1e-5 relative, so
    outside it both tracks take the same floor decision), for K = 2, 3 and 5."""
    opts, frames = _decision_track_frames()
    afl = opts.alpha_floor
    seen_k = set()
    n_pairs = 0
    for cam, fr in frames:
        S, PX, PY = _rect_pairs(cam, fr, opts)
        a32, a64 = oracle.pair_alpha(fr, S, PX, PY, opts)
        m = a64 >= 1e-3
        np.testing.assert_array_less(np.abs(a32.astype(np.float64) - a64)[m], 1e-5 * a64[m])
        clear = np.abs(a64 - afl) > 2e-5 * afl
        np.testing.assert_array_equal((a32 >= np.float32(afl))[clear], (a64 >= afl)[clear])
        tpos = fr.rec32[S, 7] > 0
        seen_k |= set(np.unique(fr.rec32[S[tpos & m], 8]).astype(int).tolist())
        n_pairs += int(m.sum())
    assert {2, 3, 5} <= seen_k
    assert n_pairs > 200_000


def test_tile_rectangle_covers_the_three_sigma_footprint():
    """The tile rectangle is the set of tiles of the square u +- r, v +- r with r = ceil(3 sqrt(
    lambda_max)) of the filtered 2D covariance (eigenvalues by numpy from the value track's conic),
    clamped to the grid; every pixel inside the 3-sigma ellipse lies in it."""
    opts, frames = _decision_track_frames()
    checked = 0
    for cam, fr in frames:
        TX, TY = oracle.tiles(cam, opts)
        for i in np.nonzero(fr.rect[:, 0] >= 0)[0]:
            v = fr.val64[i]
            conic = np.array([[v[2], v[3]], [v[3], v[4]]])
            lmax = np.linalg.eigvalsh(np.linalg.inv(conic)).max()
            r3 = 3 * math.sqrt(lmax)
            if abs(r3 - round(r3)) < 1e-4:
                continue                     # radius on an integer: fp32 and fp64 may round apart
            r = math.ceil(r3)
            e = [(v[0] - r) / opts.tile_w, (v[0] + r) / opts.tile_w, (v[1] - r) / opts.tile_h, (v[1] + r) / opts.tile_h]
            if any(abs(x - round(x)) < 1e-4 for x in e):
                continue                     # square edge on a tile boundary
            want = [max(math.floor(e[0]), 0), min(math.floor(e[1]), TX - 1),
                    max(math.floor(e[2]), 0), min(math.floor(e[3]), TY - 1)]
            assert list(fr.rect[i]) == want, (i, list(fr.rect[i]), want)
            ys, xs = np.mgrid[0:cam.height, 0:cam.width]
            dx, dy = xs + 0.5 - v[0], ys + 0.5 - v[1]
            inside = (conic[0, 0] * dx * dx + 2 * conic[0, 1] * dx * dy + conic[1, 1] * dy * dy) <= 9.0
            tx, ty = xs[inside] // opts.tile_w, ys[inside] // opts.tile_h
            assert np.all((tx >= want[0]) & (tx <= want[1]) & (ty >= want[2]) & (ty <= want[3]))
            checked += 1
    assert checked > 400
