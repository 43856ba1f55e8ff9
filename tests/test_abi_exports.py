"""The C-ABI library loads without a GPU and exports every function include/harp.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(harp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2607_12074_gb300 import _build
    return _build.build()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("harp_build_csr", "harp_select_anchors", "harp_count4", "harp_csr_free"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_exported_symbols_are_c_linkage(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(harp_\w+)\b", out))
    assert set(declared_functions()) <= exported


def test_status_strings_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.harp_status_str.restype = ctypes.c_char_p
    assert L.harp_status_str(0) == b"HARP_OK"
    assert b"invalid" in L.harp_status_str(1)


def test_argument_errors_need_no_gpu(libpath):
    """Bad arguments are rejected before any CUDA call."""
    L = ctypes.CDLL(libpath)
    out = ctypes.c_void_p()
    assert L.harp_build_csr(ctypes.c_int64(-1), ctypes.c_int64(0), None, None, 0, None, ctypes.byref(out)) == 1
    assert L.harp_build_csr(ctypes.c_int64(1 << 40), ctypes.c_int64(0), None, None, 0, None, ctypes.byref(out)) == 4
    assert L.harp_build_csr(ctypes.c_int64(5), ctypes.c_int64(3), None, None, 0, None, ctypes.byref(out)) == 1
    assert L.harp_build_csr(ctypes.c_int64(5), ctypes.c_int64(0), None, None, 7, None, ctypes.byref(out)) == 1
    assert L.harp_count4(None, None, None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2607_12074_gb300 import harp
    monkeypatch.setattr(harp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(harp, "_lib", None)
    with pytest.raises(harp.HarpUnavailable):
        harp.lib()
