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


def _c_layouts(tmp_path, structs):
    """sizeof and every field's offset of each struct, as gcc lays out include/harp.h."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "harp.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'    printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = {}
    for row in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = row.split()
        out[(s, f)] = int(v)
    return out


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the header's size and field offsets."""
    from paper_2607_12074_gb300 import harp
    classes = {name: getattr(harp, name) for name in
               ("harp_plan", "harp_select_opts", "harp_partition_stats", "harp_server_opts", "harp_server_stats")}
    structs = {name: [f for f, _ in cls._fields_] for name, cls in classes.items()}
    c = _c_layouts(tmp_path, structs)
    for name, cls in classes.items():
        assert c[(name, "size")] == ctypes.sizeof(cls), name
        for f in structs[name]:
            assert c[(name, f)] == getattr(cls, f).offset, (name, f)


def test_binding_constants_match_the_header():
    """Every HARP_* constant the binding defines has the header's value (#define or enum)."""
    from paper_2607_12074_gb300 import harp
    values = {}
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^#define\s+(HARP_\w+)\s+\(?(-?\d+)[uUlL]*\)?\s*$", text, flags=re.M):
            values[m.group(1)] = int(m.group(2))
        for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", text, flags=re.S):
            for m in re.finditer(r"(HARP_\w+)\s*=\s*(-?\d+)", body):
                values[m.group(1)] = int(m.group(2))
    bound = {k: v for k, v in vars(harp).items() if k.startswith("HARP_") and isinstance(v, int)}
    assert bound, "the binding defines no constants"
    missing = sorted(k for k in bound if k not in values)
    assert not missing, missing
    wrong = {k: (v, values[k]) for k, v in bound.items() if values[k] != v}
    assert not wrong, wrong
    # the binding's motif order is the header's HARP_<MOTIF> index order
    assert [values["HARP_" + name.upper()] for name in harp.MOTIFS] == list(range(6))
