"""CPU oracle for exact connected induced 4-vertex motif counts.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  It shares no code with the
CUDA library in ``paper_2607_12074_gb300`` and never calls it.

Functions (all take a raw undirected edge list on ids [0, n) and return numpy uint64 arrays in the
order [3-star, 4-path, tailed triangle, 4-cycle, diamond, 4-clique]):

* :func:`count4_brute`   - the definition of an induced occurrence (Section II) over every 4-subset.
* :func:`count4_esu`     - the same definition, enumerated by Wernicke's ESU.
* :func:`count4_literal` - the closure equations of Section III-F taken literally.
* :func:`count4_combo`   - plain non-induced counts (:func:`noninduced`) and the containment inversion.

Submodules (plain Python, pinned in their own tests): ``oracle.orbits`` (per-vertex orbit counts),
``oracle.edge_orbits`` (per-edge orbit counts) and ``oracle.motifs5`` (connected 5-vertex motifs).

Parity status: every function is pinned in ``tests/test_oracle_*.py`` against closed forms, brute force
and exact integer matrix identities; the paper prints no motif count, so nothing is pinned to a value
printed in the paper itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

MOTIFS = ("star3", "path4", "paw", "cycle4", "diamond", "clique4")
STATS = ("T", "K4", "C4_non", "S_non", "P_non", "paw_non", "D_non", "m")


def build(force: bool = False) -> str:
    """Compile oracle.c (plain C, OpenMP) into a shared library next to it."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32 = ctypes.c_int64, ctypes.c_int
            p32 = ctypes.POINTER(ctypes.c_int32)
            pu64 = ctypes.POINTER(ctypes.c_uint64)
            pu32 = ctypes.POINTER(ctypes.c_uint32)
            pi64 = ctypes.POINTER(ctypes.c_int64)
            lib.orc_count4_brute.argtypes = [i64, i64, p32, p32, pu64]
            for f in (lib.orc_count4_esu, lib.orc_count4_literal, lib.orc_count4_combo):
                f.argtypes = [i64, i64, p32, p32, i32, pu64]
            lib.orc_noninduced.argtypes = [i64, i64, p32, p32, i32, pu64]
            lib.orc_induced_from_noninduced.argtypes = [pu64, pu64]
            lib.orc_induced_from_noninduced.restype = None
            lib.orc_edge_triangles.argtypes = [i64, i64, p32, p32, p32, p32, pu32, i64, pi64]
            lib.orc_graph_summary.argtypes = [i64, i64, p32, p32, pi64, pi64]
            _lib = lib
    return _lib


def _edges(src, dst):
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    if s.shape != d.shape or s.ndim != 1:
        raise ValueError("src and dst must be 1-D arrays of equal length")
    return s, d


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def count4_brute(n: int, src, dst) -> np.ndarray:
    s, d = _edges(src, dst)
    out = np.zeros(6, np.uint64)
    _check(_load().orc_count4_brute(n, s.size, _ptr(s, ctypes.c_int32), _ptr(d, ctypes.c_int32),
                                    _ptr(out, ctypes.c_uint64)), "brute")
    return out


def _count(fn, what, n, src, dst, threads):
    s, d = _edges(src, dst)
    out = np.zeros(6, np.uint64)
    _check(fn(n, s.size, _ptr(s, ctypes.c_int32), _ptr(d, ctypes.c_int32), int(threads),
              _ptr(out, ctypes.c_uint64)), what)
    return out


def count4_esu(n: int, src, dst, threads: int = 0) -> np.ndarray:
    return _count(_load().orc_count4_esu, "esu", n, src, dst, threads)


def count4_literal(n: int, src, dst, threads: int = 0) -> np.ndarray:
    return _count(_load().orc_count4_literal, "literal", n, src, dst, threads)


def count4_combo(n: int, src, dst, threads: int = 0) -> np.ndarray:
    return _count(_load().orc_count4_combo, "combo", n, src, dst, threads)


def noninduced(n: int, src, dst, threads: int = 0) -> np.ndarray:
    """[T, K4, C4_non, S_non, P_non, paw_non, D_non, m] (uint64, modulo 2^64)."""
    s, d = _edges(src, dst)
    out = np.zeros(8, np.uint64)
    _check(_load().orc_noninduced(n, s.size, _ptr(s, ctypes.c_int32), _ptr(d, ctypes.c_int32), int(threads),
                                  _ptr(out, ctypes.c_uint64)), "noninduced")
    return out


def induced_from_noninduced(stats) -> np.ndarray:
    s = np.ascontiguousarray(np.asarray(stats, dtype=np.uint64))
    out = np.zeros(6, np.uint64)
    _load().orc_induced_from_noninduced(_ptr(s, ctypes.c_uint64), _ptr(out, ctypes.c_uint64))
    return out


def edge_triangles(n: int, src, dst):
    """(eu, ev, t_e) for the simple edges eu < ev in lexicographic order; t_e = |N(u) n N(v)|."""
    s, d = _edges(src, dst)
    cap = max(1, s.size)
    eu = np.zeros(cap, np.int32)
    ev = np.zeros(cap, np.int32)
    te = np.zeros(cap, np.uint32)
    m = ctypes.c_int64(0)
    _check(_load().orc_edge_triangles(n, s.size, _ptr(s, ctypes.c_int32), _ptr(d, ctypes.c_int32),
                                      _ptr(eu, ctypes.c_int32), _ptr(ev, ctypes.c_int32),
                                      _ptr(te, ctypes.c_uint32), cap, ctypes.byref(m)), "edge_triangles")
    k = m.value
    return eu[:k], ev[:k], te[:k]


def graph_summary(n: int, src, dst):
    """(m undirected simple edges, max degree)."""
    s, d = _edges(src, dst)
    m = ctypes.c_int64(0)
    md = ctypes.c_int64(0)
    _check(_load().orc_graph_summary(n, s.size, _ptr(s, ctypes.c_int32), _ptr(d, ctypes.c_int32),
                                     ctypes.byref(m), ctypes.byref(md)), "summary")
    return m.value, md.value
