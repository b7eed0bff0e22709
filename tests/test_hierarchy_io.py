"""Hierarchy files: a round trip keeps every array bit-exact, and broken files are refused."""
import numpy as np
import pytest

import oracle
from paper_2406_12080_b300 import hierarchy_io
from tests import scenes


def test_round_trip_is_bit_exact(tmp_path):
    _, h = scenes.tiny()
    p = tmp_path / "h.npz"
    hierarchy_io.save_hierarchy(str(p), h)
    g = hierarchy_io.load_hierarchy(str(p))
    for k in hierarchy_io.FLOAT_KEYS + hierarchy_io.INT_KEYS:
        np.testing.assert_array_equal(g[k], getattr(h, k), err_msg=k)
    # the loaded arrays render the same cut with the oracle
    sc, _ = scenes.tiny()
    h2 = oracle.Hierarchy(**{k: g[k] for k in hierarchy_io.FLOAT_KEYS + hierarchy_io.INT_KEYS})
    a, _ = oracle.select_cut(sc.cameras[0], h, 1)
    b, _ = oracle.select_cut(sc.cameras[0], h2, 1)
    np.testing.assert_array_equal(a, b)


def test_broken_topology_and_versions_are_refused(tmp_path):
    _, h = scenes.tiny()
    p = tmp_path / "h.npz"
    hierarchy_io.save_hierarchy(str(p), h)
    good = dict(np.load(str(p)))
    for name, edit in (("version", lambda d: d.update(version=np.int64(99))),
                       ("parent", lambda d: d["parent"].__setitem__(5, 7)),
                       ("child", lambda d: d["child_start"].__setitem__(0, 3)),
                       ("shape", lambda d: d.update(sh=d["sh"][:, :12]))):
        d = {k: v.copy() for k, v in good.items()}
        edit(d)
        q = tmp_path / f"bad_{name}.npz"
        np.savez(str(q), **d)
        with pytest.raises(ValueError):
            hierarchy_io.load_hierarchy(str(q))
