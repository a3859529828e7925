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
              "dexel_offset_batched", "dexel_workspace_size", "dexel_validate",
              "dexel_status_string"]:
        assert s in syms


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
