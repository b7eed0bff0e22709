"""Pins of the oracle's chunk consolidation (Sec. 6.3; reading 16): chunk hierarchies joined by a top
tree over the chunk roots.  Checked against facts outside the consolidation code: a single chunk is
returned unchanged; every chunk's subtree is its own hierarchy, relabelled; the top tree is a
median-split BVH whose boxes are unions; every top-tree node is the moment-matched Gaussian of its two
children (mixture mean and covariance by the law of total variance, written here in numpy, with the
weights o_i S_i of Eq. merge)."""
import numpy as np
import pytest

import oracle
from tests import scenes
from tests.test_oracle_pins import _cov


def _chunks(K, seed=4, per=24):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(K):
        lv, _ = scenes.small_random_scene(n_leaves=per, seed=seed + k, cube=2.0)
        lv.mean[:] += np.float32(rng.uniform(-20, 20, 3))
        out.append(oracle.build_tree(lv))
    return out


def _descendants(h, v):
    out, stack = [], [v]
    while stack:
        u = stack.pop()
        out.append(u)
        if h.child_count[u] > 0:
            stack.extend(range(h.child_start[u], h.child_start[u] + h.child_count[u]))
    return np.sort(np.array(out))


def test_single_chunk_is_unchanged():
    h = _chunks(1)[0]
    c = oracle.consolidate([h])
    for k in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "parent", "child_start", "child_count"):
        np.testing.assert_array_equal(getattr(c, k), getattr(h, k), err_msg=k)


@pytest.mark.parametrize("K", [2, 5, 16])
def test_consolidated_tree(K):
    chunks = _chunks(K)
    c = oracle.consolidate(chunks)
    n_top = 2 * K - 1
    assert c.n == n_top + sum(h.n - 1 for h in chunks)
    # breadth-first, children contiguous, parent < child
    assert c.parent[0] == -1
    for v in range(c.n):
        if c.child_count[v]:
            kids = np.arange(c.child_start[v], c.child_start[v] + c.child_count[v])
            assert np.all(c.parent[kids] == v) and np.all(kids > v)
    # the top tree's leaves are the chunk roots: each one's subtree is its chunk, rows and boxes unchanged
    roots = [v for v in range(n_top) if c.child_start[v] >= n_top or c.child_count[v] == 0]
    assert len(roots) == K
    for v in roots:
        sub = _descendants(c, v)
        k = [i for i, h in enumerate(chunks) if h.n == len(sub) and np.array_equal(c.mean[v], h.mean[0])]
        assert len(k) == 1
        h = chunks[k[0]]
        # breadth-first order within the chunk is kept: subtree = root, then the chunk's nodes 1..
        order = np.concatenate([[v], sub[sub != v]])
        for key in ("mean", "scale", "rot", "opacity", "sh", "box_min", "box_max", "child_count"):
            np.testing.assert_array_equal(getattr(c, key)[order], getattr(h, key), err_msg=key)
    # top-tree interior nodes: union boxes, median split, moment-matched merge of the two children
    for v in range(n_top):
        if v in roots:
            continue
        a, b = c.child_start[v], c.child_start[v] + 1
        np.testing.assert_array_equal(c.box_min[v], np.minimum(c.box_min[a], c.box_min[b]))
        np.testing.assert_array_equal(c.box_max[v], np.maximum(c.box_max[a], c.box_max[b]))
        axis = int(np.argmax(c.box_max[v].astype(np.float64) - c.box_min[v].astype(np.float64)))
        lr = [[u for u in roots if np.isin(u, _descendants(c, side))] for side in (a, b)]
        assert abs(len(lr[0]) - len(lr[1])) <= 1 and len(lr[0]) <= len(lr[1])
        assert max(c.mean[u, axis] for u in lr[0]) <= min(c.mean[u, axis] for u in lr[1])
        w = np.array([c.opacity[u] * oracle.ellipsoid_area(c.scale[u]) for u in (a, b)], np.float64)
        w /= w.sum()
        mu = [c.mean[u].astype(np.float64) for u in (a, b)]
        m = w[0] * mu[0] + w[1] * mu[1]
        S = sum(w[i] * (_cov(c.scale[u], c.rot[u]) + np.outer(mu[i] - m, mu[i] - m)) for i, u in enumerate((a, b)))
        np.testing.assert_allclose(c.mean[v], m, rtol=1e-6, atol=1e-5)
        np.testing.assert_allclose(_cov(c.scale[v], c.rot[v]), S, rtol=2e-5, atol=1e-6 * np.abs(S).max())
        np.testing.assert_allclose(c.sh[v], w[0] * c.sh[a] + w[1] * c.sh[b], rtol=1e-5, atol=1e-6)
