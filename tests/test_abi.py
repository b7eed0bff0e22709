"""The C-ABI library loads on a machine without a GPU and exports every declared entry point."""
import ctypes as C

import pytest

from paper_2406_12080_b300 import build, h3dgs


@pytest.fixture(scope="module")
def L():
    build.build()
    return h3dgs.lib()


def test_every_declared_symbol_is_exported(L):
    names = h3dgs.header_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    for required in ("h3dgs_upload_hierarchy", "h3dgs_select_cut", "h3dgs_interpolate", "h3dgs_render",
                     "h3dgs_render_backward"):
        assert required in names


def test_default_opts(L):
    o = h3dgs.default_opts()
    assert (o.tile_w, o.tile_h) == (16, 16)
    assert o.lowpass == pytest.approx(0.3)
    assert o.alpha_clamp == pytest.approx(0.99)
    assert o.alpha_floor == pytest.approx(1 / 255)
    assert o.t_min == pytest.approx(1e-4)
    assert (o.aa_compensate, o.interpolate) == (1, 1)


def test_null_context_and_no_device(L):
    assert L.h3dgs_destroy(None) == 0
    assert L.h3dgs_last_error(None) == b"null context"
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = C.c_void_p()
    assert L.h3dgs_create(C.byref(out), 0, None) == 7   # H3DGS_ERR_NO_DEVICE
    assert not out.value
