"""The calibration kernels behind the roofline denominators give rates within the B300's unit
counts: fp32 at most 148 SMs x 128 lanes x 2 flops x 2.032 GHz (77 TFLOP/s) and at least a third of
it; exp2 at least 148 SMs x 16 per clock / 10 and at most 148 x 32 per clock x 2.032 GHz (this part
raised the special-function rate for exponentials above the 16 per SM and clock of earlier parts)."""
import pytest

from paper_2406_12080_b300 import h3dgs

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_within_the_unit_count_bounds():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    build.build()
    ctx = h3dgs.Context(torch.cuda.current_device())
    try:
        p = h3dgs.h3dgs_measure_peaks(ctx.ctx)
    finally:
        ctx.close()
    nominal_fp32 = 148 * 128 * 2 * 2.032e9 / 1e12
    ex2_16 = 148 * 16 * 2.032e9 / 1e9
    assert nominal_fp32 / 3 < p["fp32_tflops"] <= nominal_fp32 * 1.02, p
    assert ex2_16 / 10 < p["ex2_gops"] <= 2 * ex2_16 * 1.02, p
