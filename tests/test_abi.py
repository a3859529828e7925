"""The C ABI library builds, loads and exports every entry point declared in include/dexel.h.

No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dexel.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dexel_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1804_08968_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["dexel_ctx_create", "dexel_ctx_destroy", "dexel_dilate", "dexel_erode",
              "dexel_morph", "dexel_offset_batched", "dexel_workspace_size", "dexel_validate",
              "dexel_status_string", "dexel_boolean", "dexel_shell", "dexel_offset_slices",
              "dexel_raycast", "dexel_raycast_axis", "dexel_offset_ldi", "dexel_offset_noalloc"]:
        assert s in syms


def test_entry_points_reject_missing_arguments(libpath):
    """Every compute entry point returns DEXEL_ERR_INVALID_ARG for a null context or output
    before touching the device (host-side checks only)."""
    import paper_1804_08968_gb300 as dx
    L = dx.lib()
    P = ctypes.c_void_p
    gin = dx._In(4, 4, 0.1, 1, 1, 0)
    out = dx._Out(1, 1, 10, 0)
    assert L.dexel_dilate(None, ctypes.byref(gin), 1.0, 0, ctypes.byref(out), None, 0, None) == -1
    assert L.dexel_boolean(None, 0, ctypes.byref(gin), ctypes.byref(gin), 0, ctypes.byref(out),
                           None, 0, None) == -1
    assert L.dexel_shell(None, ctypes.byref(gin), 1.0, 0, ctypes.byref(out), None, 0, None) == -1
    assert L.dexel_offset_slices(None, ctypes.byref(gin), 1.0, 0, 0, ctypes.byref(out), None, 0,
                                 None) == -1
    assert L.dexel_raycast_axis(None, None, 0, 2, 4, 4, 0.25, 0, ctypes.byref(out), None, 0,
                                None) == -1
    assert L.dexel_offset_ldi(None, None, 1.0, 0, 0, None, None, 0, None) == -1
    assert L.dexel_offset_enqueue(None, ctypes.byref(gin), 1.0, 0, 0, ctypes.byref(out), None, 0,
                                  None, None) == -1
    # a bad operation is refused the same way
    assert L.dexel_offset_slices(None, ctypes.byref(gin), 1.0, 7, 0, ctypes.byref(out), None, 0,
                                 None) == -1


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings(libpath):
    lib = ctypes.CDLL(libpath)
    lib.dexel_status_string.restype = ctypes.c_char_p
    lib.dexel_status_string.argtypes = [ctypes.c_int]
    assert lib.dexel_status_string(0) == b"ok"
    assert b"CSR" in lib.dexel_status_string(-2)
    assert lib.dexel_status_string(-99) == b"unknown status"
    assert b"plan" in lib.dexel_status_string(-7)


def test_workspace_size_rejects_bad_input(libpath):
    import paper_1804_08968_gb300 as dx
    L = dx.lib()
    gin = dx._In(0, 4, 0.1, None, None, 0)
    assert L.dexel_workspace_size(ctypes.byref(gin), 2.0, 0) == 0
    gin = dx._In(4, 4, 0.1, 1, 1, 0)
    assert L.dexel_workspace_size(ctypes.byref(gin), -1.0, 0) == 0
    assert L.dexel_workspace_size(ctypes.byref(gin), 2.0, 0) > 0


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    import paper_1804_08968_gb300 as dx
    monkeypatch.setattr(dx, "_lib", None)
    monkeypatch.setattr(dx, "_LIBPATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        dx.lib()
