"""Behaviour tied to the numbers the paper states (tests/golden/paper_constants.txt): the alpha clamp of
the blend, and the granularity range of compaction and hierarchy optimisation."""
import os

import numpy as np

import oracle
from paper_2406_12080_b300 import synth
from tests import scenes

_HERE = os.path.dirname(os.path.abspath(__file__))


def _constants():
    out = {}
    for line in open(os.path.join(_HERE, "golden", "paper_constants.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_an_opaque_splat_is_clamped_at_its_centre():
    """A splat of opacity 1 at a pixel centre blends with alpha = the clamp: T_final = 1 - clamp."""
    c = _constants()["alpha_clamp"]
    lv = scenes.leaves_from([[0.0, 0.0, 3.0]], [[0.2, 0.2, 0.2]], [[1.0, 0.0, 0.0, 0.0]], [1.0])
    h = oracle.build_tree(lv)
    cam = scenes.axis_camera(16, 16, 40.0, cx=8.5, cy=8.5)
    fr = oracle.render(cam, h, oracle.Opts(aa_compensate=0))
    assert abs(fr.T_final[8, 8] - (1.0 - np.float32(c))) < 1e-7
    assert oracle.Opts().alpha_clamp == np.float32(c)


def test_optimisation_granularities_span_the_stated_range():
    c = _constants()
    _, views = synth.optimisation_views(n_views=64, width=1280)
    taus = np.array([v.tau for v in views])
    assert taus.min() >= c["tau_min_px"] and taus.max() < c["tau_max_fraction_of_width"] * 1280
    assert taus.min() < 2 * c["tau_min_px"] and taus.max() > 0.25 * c["tau_max_fraction_of_width"] * 1280
