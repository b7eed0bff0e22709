"""Pins of the oracle's hierarchy compaction (Sec. 5.2) against results fixed by other routes:
a brute-force restatement over explicit descendant sets with the recursive-descent cut, the
closed form of the kept set, and the special cases that reduce to known trees."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import synth
from tests import scenes


def _levels(tau_min, tau_max):
    out, t = [], np.float32(tau_min)
    while t <= np.float32(tau_max):
        out.append(t)
        t = np.float32(t * np.float32(2.0))
    return out


def _children(h):
    return [list(range(h.child_start[v], h.child_start[v] + h.child_count[v])) for v in range(h.n)]


def _brute_force(cams, h, tau_min, tau_max):
    """The paper's procedure with sets: cuts by recursive descent, descendants enumerated."""
    kids = _children(h)
    desc = [None] * h.n
    for v in range(h.n - 1, -1, -1):
        desc[v] = set(kids[v]).union(*[desc[c] for c in kids[v]]) if kids[v] else set()
    marked = {v for v in range(h.n) if h.child_count[v] == 0}
    removed = set()
    for tau in _levels(tau_min, tau_max):
        union = set()
        for cam in cams:
            union |= set(oracle.select_cut_descent(synth.with_tau(cam, float(tau)), h).tolist())
        bottom = {u for u in union if not (desc[u] & union)}
        strictly_below = set().union(*[desc[b] for b in bottom])
        removed |= strictly_below - marked
        marked |= bottom
    kept = sorted(set(range(h.n)) - removed)
    # closest kept ancestor, then breadth-first order with siblings by old index
    up = {}
    for v in kept[1:]:
        p = int(h.parent[v])
        while p in removed:
            p = int(h.parent[p])
        up[v] = p
    order = [0]
    for o in order:
        order += sorted(v for v in kept[1:] if up[v] == o)
    return order, up


@pytest.fixture(scope="module")
def small():
    lv, _ = scenes.small_random_scene(n_leaves=40, seed=11, cube=1.0, dist=3.0)
    h = oracle.build_tree(lv)
    cams = synth.orbit_views([0.0, 0.0, 3.0], 3.5, 3, 64, 48, seed=1)
    return h, cams


@pytest.mark.parametrize("tau_min,tau_max", [(1.0, 64.0), (0.5, 8.0), (3.0, 32.0)])
def test_matches_the_brute_force_procedure(small, tau_min, tau_max):
    h, cams = small
    out, old = oracle.compact(cams, h, tau_min, tau_max)
    order, up = _brute_force(cams, h, tau_min, tau_max)
    assert old.tolist() == order
    new_of_old = {o: i for i, o in enumerate(order)}
    assert out.parent[0] == -1
    assert [int(p) for p in out.parent[1:]] == [new_of_old[up[o]] for o in order[1:]]



@pytest.mark.parametrize("seed", range(8))
def test_matches_the_brute_force_procedure_on_random_trees(seed):
    """The same equality on seeded random trees (5 to 80 leaves), camera sets (1 to 4 orbit views at
    random distances) and tau ranges drawn inside the interior nodes' granularities (so that nodes
    are removed and wider nodes made)."""
    rng = np.random.default_rng([seed, 31])
    n_leaves = int(rng.choice([5, 17, 40, 80]))
    lv, _ = scenes.small_random_scene(n_leaves=n_leaves, seed=500 + seed, cube=1.0, dist=3.0)
    h = oracle.build_tree(lv)
    cams = synth.orbit_views([0.0, 0.0, 3.0], float(rng.uniform(2.0, 8.0)), int(rng.integers(1, 5)), 64, 48,
                             seed=int(rng.integers(1000)))
    eps = np.concatenate([oracle.granularity(c, h)[h.child_count > 0] for c in cams])
    tau_min = float(np.quantile(eps[np.isfinite(eps)], rng.uniform(0.05, 0.6)))
    tau_max = tau_min * float(2 ** rng.integers(1, 6))
    out, old = oracle.compact(cams, h, tau_min, tau_max)
    order, up = _brute_force(cams, h, tau_min, tau_max)
    assert old.tolist() == order
    new_of_old = {o: i for i, o in enumerate(order)}
    assert out.parent[0] == -1
    assert [int(p) for p in out.parent[1:]] == [new_of_old[up[o]] for o in order[1:]]

def test_brute_force_case_removes_nodes_and_makes_wider_nodes(small):
    h, cams = small
    out, old = oracle.compact(cams, h, 1.0, 64.0)
    assert out.n < h.n
    assert out.child_count.max() > 2


@pytest.fixture(scope="module")
def tiny_compacted():
    sc, h = scenes.tiny()
    cams = synth.orbit_views([5.0, 5.0, 5.0], 14.0, 12, 256, 256, seed=2)
    out, old = oracle.compact(cams, h, 3.0, 128.0)
    return h, cams, out, old


def test_kept_set_has_the_closed_form(tiny_compacted):
    """Granularity never decreases towards the root, so with e(n) = max over the views of eps(n) the
    union's bottom-most nodes at tau are the nodes with (leaf or e(n) < tau) and (root or
    e(parent) >= tau), and a node lies strictly below one of them iff e(parent) < tau.  Hence a node
    survives iff it is a leaf or the root, or e(parent) >= the last level, or some level tau_k has
    e(n) < tau_k <= e(parent)."""
    h, cams, out, old = tiny_compacted
    e = np.max(np.stack([oracle.granularity(c, h) for c in cams]), axis=0)
    lv = _levels(3.0, 128.0)
    ep = np.where(h.parent >= 0, e[np.maximum(h.parent, 0)], np.inf)
    straddle = np.zeros(h.n, bool)
    for t in lv:
        straddle |= (e < t) & (t <= ep)
    keep = (h.child_count == 0) | (h.parent < 0) | (ep >= lv[-1]) | straddle
    assert sorted(old.tolist()) == np.flatnonzero(keep).tolist()
    assert out.n < h.n and out.child_count.max() > 2


def test_compacted_tree_is_a_breadth_first_tree_of_closest_kept_ancestors(tiny_compacted):
    h, cams, out, old = tiny_compacted
    n = out.n
    kept = set(old.tolist())
    leaves_before = set(np.flatnonzero(h.child_count == 0).tolist())
    assert leaves_before <= kept
    assert set(old[out.child_count == 0].tolist()) == leaves_before
    assert out.parent[0] == -1 and np.all(out.parent[1:] < np.arange(1, n))
    depth = np.zeros(n, np.int64)
    for i in range(1, n):
        depth[i] = depth[out.parent[i]] + 1
    assert np.all(np.diff(depth) >= 0)
    for i in range(n):
        c0, k = out.child_start[i], out.child_count[i]
        if k == 0:
            assert c0 == -1
            continue
        assert k >= 2
        assert np.all(out.parent[c0:c0 + k] == i)
        assert np.all(np.diff(old[c0:c0 + k]) > 0)
        # every child's old ancestors below i were removed
        for c in old[c0:c0 + k]:
            p = int(h.parent[c])
            while p != old[i]:
                assert p not in kept
                p = int(h.parent[p])
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max"):
        np.testing.assert_array_equal(getattr(out, k), getattr(h, k)[old])


def test_tau_min_above_every_granularity_leaves_root_and_leaves():
    sc, h = scenes.tiny()
    far = synth.look_camera([5.0, 5.0, -2.0e4], [0, 0, 1], [0, -1, 0], 256, 256, 60.0, 6.0)
    e_root = oracle.granularity(far, h)[0]
    assert e_root < 3.0
    out, old = oracle.compact([far], h, 3.0, 128.0)
    leaves = np.flatnonzero(h.child_count == 0)
    assert out.n == 1 + len(leaves)
    assert old[0] == 0 and old[1:].tolist() == leaves.tolist()
    assert out.child_count[0] == len(leaves) and out.child_start[0] == 1


def test_no_level_leaves_the_tree_unchanged():
    sc, h = scenes.tiny()
    out, old = oracle.compact(sc.cameras, h, 8.0, 4.0)
    np.testing.assert_array_equal(old, np.arange(h.n))
    for k in ("parent", "child_start", "child_count"):
        np.testing.assert_array_equal(getattr(out, k), getattr(h, k))
