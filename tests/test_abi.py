"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(stencil_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1410_5561_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # pragma: no cover - toolkit missing
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["stencil_create", "stencil_set_coeffs", "stencil_set_field", "stencil_run",
              "stencil_get_field", "stencil_destroy", "stencil_strerror"]:
        assert n in names


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1410_5561_gb300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert _declared() <= bound, _declared() - bound


def test_host_only_entry_points(libpath):
    """Entry points that touch no device memory run on a CPU-only machine."""
    from paper_1410_5561_gb300 import _lib
    L = _lib.lib()
    assert L.stencil_strerror(0) == b"ok"
    assert L.stencil_strerror(-2).startswith(b"blocked tuning")
    h = ctypes.c_void_p()
    assert L.stencil_create(ctypes.byref(h), 0, 0, 4, 4, 0, 0, None) == -1   # empty grid
    assert L.stencil_create(ctypes.byref(h), 3, 4, 4, 4, 0, 0, None) == -1   # bad kind
    assert L.stencil_create(ctypes.byref(h), 1, 4, 4, 4, 1, 2, None) == -1   # BF16 coef needs FP32 field
    assert L.stencil_create(ctypes.byref(h), 2, 100, 30, 20, 0, 2, None) == 0
    lay = _lib.stencil_layout()
    assert L.stencil_layout_of(h, 0, ctypes.byref(lay)) == 0
    assert lay.radius == 4 and lay.x_offset % 4 == 0 and lay.x_offset >= 4
    assert lay.pitch_x >= lay.x_offset + 100 + 4 and (lay.pitch_x * 4) % 128 == 0
    assert lay.pitch_y == 38 and lay.planes == 28
    assert lay.bytes == lay.pitch_x * lay.pitch_y * lay.planes * 4
    assert L.stencil_layout_of(h, 1, ctypes.byref(lay)) == 0 and lay.elem_bytes == 2
    assert L.stencil_run(h, 1) == -5      # nothing bound yet
    assert L.stencil_run(h, -1) == -1
    assert L.stencil_bind(h, ctypes.c_void_p(16), ctypes.c_void_p(16), None, None) == -1
    assert L.stencil_bind(h, ctypes.c_void_p(18), ctypes.c_void_p(32), None, None) == -1
    assert L.stencil_destroy(h) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the CUDA library every entry point raises; nothing falls back to the CPU."""
    from paper_1410_5561_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libstencil_gb300.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.call("stencil_strerror", 0)


def test_sm_copy_refuses_memory_the_device_cannot_address():
    """stencil_copy checks both pointers before any access: plain host memory (here no GPU at
    all, or pageable memory on a GPU machine) is refused with STENCIL_EINVAL."""
    import ctypes
    from paper_1410_5561_gb300 import _lib as C
    buf = (ctypes.c_char * 64)()
    r = C.lib().stencil_copy(ctypes.c_void_p(ctypes.addressof(buf)), ctypes.c_void_p(ctypes.addressof(buf)),
                             ctypes.c_size_t(64), 4, None)
    assert C.STATUS[r] == "STENCIL_EINVAL"
