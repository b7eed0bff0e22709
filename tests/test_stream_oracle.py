"""Pins of the oracle's streaming residency trace (Sec. 6.3) by set arithmetic that does not go
through the trace: transfers of a static camera, the union of the needed sets without cleanup, and
the residents after an aggressive cleanup."""
import numpy as np

import oracle
from paper_2406_12080_b300 import synth
from tests import scenes


def _path(n):
    return synth.orbit_views([5.0, 5.0, 5.0], 14.0, n, 128, 128, tau=4.0, seed=3)


def _needed(cam, h):
    ids, t = oracle.select_cut(cam, h)
    p = h.parent[ids]
    return set(ids.tolist()) | set(p[(t != 0) & (p >= 0)].tolist())


def test_static_camera_transfers_once():
    sc, h = scenes.tiny()
    cams = [sc.cameras[0]] * 7
    tr, _, res = oracle.stream_trace(cams, h, update_every=2, cleanup_every=100)
    need = _needed(sc.cameras[0], h)
    assert tr == [len(need), 0, 0, 0] and res == len(need)


def test_without_cleanup_every_needed_node_is_transferred_exactly_once():
    sc, h = scenes.tiny()
    cams = _path(12)
    tr, _, res = oracle.stream_trace(cams, h, update_every=2, cleanup_every=1000)
    union = set().union(*[_needed(c, h) for c in cams[::2]])
    assert sum(tr) == len(union) == res
    assert tr[0] == len(_needed(cams[0], h)) and min(tr[1:]) > 0


def test_cleanup_with_zero_age_keeps_only_the_last_update():
    sc, h = scenes.tiny()
    cams = _path(8)
    tr, after, res = oracle.stream_trace(cams, h, update_every=2, cleanup_every=2, max_age=1)
    # cleanup after frames 1, 3, 5, 7 keeps what the update at frames 0, 2, 4, 6 stamped
    assert after == [len(_needed(cams[f], h)) for f in (0, 2, 4, 6)]
    # each update after a cleanup transfers what the previous update did not need
    for k in range(1, 4):
        assert tr[k] == len(_needed(cams[2 * k], h) - _needed(cams[2 * k - 2], h))
