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


def test_concurrent_builds_compile_once(tmp_path, monkeypatch):
    """Two callers of build() at once (every rank of a multi-GPU run calls it) while the library is
    missing: one compiles and links, the other waits for the build folder's lock, then finds the
    library fresh and returns it (the compiler is replaced by a stub that writes its output)."""
    import threading
    import time
    lib = tmp_path / "libh3dgs.so"
    monkeypatch.setattr(build, "LIB", str(lib))
    monkeypatch.setattr(build, "BUILD_DIR", str(tmp_path / "_build"))
    monkeypatch.setattr(build, "nvcc", lambda: "nvcc")
    links, errors = [], []

    def stub(cmd):
        out = cmd[cmd.index("-o") + 1]
        if "-shared" in cmd:
            links.append(out)
            time.sleep(0.3)   # the other caller arrives while this one links
        with open(out, "w") as f:
            f.write("stub")
        return 0

    monkeypatch.setattr(build.subprocess, "check_call", stub)

    def call():
        try:
            assert build.build() == str(lib)
        except Exception as e:   # reported below
            errors.append(e)

    threads = [threading.Thread(target=call) for _ in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert len(links) == 1 and lib.exists()
