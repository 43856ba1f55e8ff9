"""Seeded synthetic graph generators shared by the oracle tests, the GPU tests and bench.py.

This package draws undirected edge lists and nothing else: it contains none of the motif-counting
arithmetic.  The paper evaluates on social, web, biological and synthetic R-MAT graphs (Section IV-B,
Table I); those datasets are not available here, so these generators stand in for the families:

* Barabasi-Albert (social-like skew), R-MAT (a=0.57, b=0.19, c=0.19, d=0.05; social/synthetic skew),
* Erdos-Renyi (unskewed control), random geometric 2-D (localised, low degree: the biological stand-in),
* Chung-Lu power law (web-like heavy tail).

All randomness is SplitMix64 implemented in ``graphgen.c`` so a seed yields the same bytes on x86-64
and AArch64.  Edge lists may contain self-loops and duplicates (R-MAT, Chung-Lu); every consumer drops
them when it builds its own adjacency.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library next to it (host C only, no GPU code)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            p32 = ctypes.POINTER(ctypes.c_int32)
            lib.gg_ba.argtypes = [i64, i32, u64, p32, p32, i64]
            lib.gg_er.argtypes = [i64, dbl, u64, p32, p32, i64]
            lib.gg_rgg.argtypes = [i64, dbl, u64, p32, p32, i64]
            lib.gg_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, p32, p32, i64]
            lib.gg_chung_lu.argtypes = [i64, dbl, dbl, dbl, u64, i64, i64, p32, p32, i64]
            lib.gg_chung_lu_induced.argtypes = [i64, dbl, dbl, dbl, u64, p32, i64, i64, i64, p32, p32, i64]
            lib.gg_splitmix64_at.argtypes = [u64, u64, i64]
            for f in (lib.gg_ba, lib.gg_er, lib.gg_rgg, lib.gg_rmat, lib.gg_chung_lu, lib.gg_chung_lu_induced):
                f.restype = i64
            lib.gg_splitmix64_at.restype = u64
            _lib = lib
    return _lib


@dataclass
class Graph:
    """An undirected edge list on vertex ids [0, n).  May hold duplicates and self-loops."""
    n: int
    src: np.ndarray  # int32[m_in]
    dst: np.ndarray  # int32[m_in]
    name: str = ""

    @property
    def m_in(self) -> int:
        return int(self.src.shape[0])


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _call_growing(fn, args, cap: int):
    while True:
        src = np.empty(max(cap, 1), np.int32)
        dst = np.empty(max(cap, 1), np.int32)
        got = fn(*args, _p(src), _p(dst), cap)
        if got >= 0:
            return src[:got].copy(), dst[:got].copy()
        cap = int(-got) + 16


def splitmix64_at(seed: int, purpose: int, index: int) -> int:
    return int(_load().gg_splitmix64_at(seed, purpose, index))


def ba(n: int, m: int, seed: int) -> Graph:
    """Barabasi-Albert graph, seed clique K_{m+1}, m edges per new vertex."""
    k0 = min(n, m + 1)
    cap = k0 * (k0 - 1) // 2 + max(0, n - k0) * m
    src, dst = _call_growing(_load().gg_ba, (n, m, seed), cap)
    return Graph(n, src, dst, f"ba(n={n},m={m},seed={seed})")


def er(n: int, mean_degree: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, p) with p = k / (n - 1)."""
    p = min(1.0, mean_degree / max(1, n - 1))
    cap = int(n * mean_degree / 2 * 1.2) + 64
    src, dst = _call_growing(_load().gg_er, (n, p, seed), cap)
    return Graph(n, src, dst, f"er(n={n},k={mean_degree:g},seed={seed})")


def rgg_radius(n: int, mean_degree: float) -> float:
    """Radius giving expected degree k in the unit square, ignoring the boundary: pi r^2 (n-1) = k."""
    return math.sqrt(mean_degree / (math.pi * max(1, n - 1)))


def rgg(n: int, mean_degree: float, seed: int) -> Graph:
    """Random geometric graph in the unit square (no torus), radius from the target mean degree."""
    r = rgg_radius(n, mean_degree)
    cap = int(n * mean_degree / 2 * 1.2) + 64
    src, dst = _call_growing(_load().gg_rgg, (n, r, seed), cap)
    return Graph(n, src, dst, f"rgg(n={n},k={mean_degree:g},seed={seed})")


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1) -> Graph:
    """R-MAT with ef * 2^scale draws, then a seeded vertex permutation.  d = 1 - a - b - c."""
    n = 1 << scale
    src, dst = _call_growing(_load().gg_rmat, (scale, edge_factor, a, b, c, seed), edge_factor * n)
    return Graph(n, src, dst, f"rmat(scale={scale},ef={edge_factor},seed={seed})")


def _chung_lu_scale(n: int, gamma: float, max_weight: float, mean_degree: float):
    """(c, i0) with w_0 = c i0^(-1/(gamma-1)) = max_weight and sum_i w_i ~= n * mean_degree."""
    ex = -1.0 / (gamma - 1.0)
    target = n * mean_degree

    def total(i0):
        c = max_weight * i0 ** (-ex)
        # integral approximation of sum_{i<n} (i+i0)^ex, plus the first term exactly
        s = ((n - 1 + i0) ** (ex + 1) - i0 ** (ex + 1)) / (ex + 1) + i0 ** ex
        return c * s

    lo, hi = 1e-6, float(n)
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if total(mid) > target:
            hi = mid
        else:
            lo = mid
    i0 = math.sqrt(lo * hi)
    return max_weight * i0 ** (-ex), i0


def chung_lu(n: int, gamma: float, max_weight: float, mean_degree: float, seed: int,
             rows: tuple[int, int] | None = None) -> Graph:
    """Chung-Lu power law with w_i = c (i + i0)^(-1/(gamma-1)).

    c and i0 are fixed so that w_0 = max_weight and sum_i w_i ~= n * mean_degree (bisection on i0).
    ``rows`` restricts sampling to pair rows [lo, hi) (for chunked generation of very large graphs).
    """
    c, i0 = _chung_lu_scale(n, gamma, max_weight, mean_degree)
    ex = -1.0 / (gamma - 1.0)
    name = f"chung_lu(n={n},gamma={gamma},seed={seed})"
    if rows is None and n >= 1_000_000:
        # every row draws from its own stream, so row chunks are independent: generate balanced
        # chunks on threads (the C call releases the interpreter lock) and concatenate in row order
        import threading
        w = c * np.power(np.arange(n, dtype=np.float64) + i0, ex)
        S = float(w.sum())
        tail = np.cumsum(w[::-1])[::-1] - w                       # sum_{v > u} w_v
        expect = np.minimum(w * tail / S, np.arange(n, 0, -1) - 1.0)  # expected edges of row u
        cum = np.cumsum(expect)
        parts = max(1, min(64, (os.cpu_count() or 4) * 2))
        cuts = [0] + [int(np.searchsorted(cum, cum[-1] * k / parts)) for k in range(1, parts)] + [n]
        cuts = sorted(set(cuts))
        out = [None] * (len(cuts) - 1)

        def work(k):
            a, b = cuts[k], cuts[k + 1]
            est = float(cum[b - 1] - (cum[a - 1] if a > 0 else 0.0))
            cap = int(est * 1.05 + 6 * math.sqrt(est + 1)) + 1024
            out[k] = _call_growing(_load().gg_chung_lu, (n, gamma, c, i0, seed, a, b), cap)

        th = [threading.Thread(target=work, args=(k,)) for k in range(len(out))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        return Graph(n, np.concatenate([o[0] for o in out]), np.concatenate([o[1] for o in out]), name)
    r0, r1 = rows if rows is not None else (0, n)
    cap = int((r1 - r0) * mean_degree * 0.6) + 1024
    src, dst = _call_growing(_load().gg_chung_lu, (n, gamma, c, i0, seed, r0, r1), cap)
    return Graph(n, src, dst, name)


# ---------------------------------------------------------------------------------------------
# The named workloads.
# ---------------------------------------------------------------------------------------------

def ba_2000() -> Graph:
    """Plain single graph: Barabasi-Albert, n = 2,000, 4 edges per new vertex, seed 1 (~8k edges)."""
    return ba(2000, 4, 1)


def rmat_scale20() -> Graph:
    """Plain single large skewed graph: R-MAT scale 20, edge factor 16, (0.57, 0.19, 0.19, 0.05), seed 1."""
    return rmat(20, 16, 0.57, 0.19, 0.19, seed=1)


@dataclass
class BatchSpec:
    seed: int
    kind: str      # "er" | "ba" | "rgg"
    n: int
    k: float       # mean degree (er, rgg)
    m: int         # edges per new vertex (ba)


def chung_lu_large(n: int = 50_000_000, seed: int = 1) -> Graph:
    """The partitioned large-graph workload: Chung-Lu, exponent 2.1, max expected degree 1e6, mean
    degree 48 (about 1.2e9 edges at n = 5e7).  Smaller n keeps the shape for trial runs."""
    return chung_lu(n, 2.1, 1e6 * n / 50_000_000, 48.0, seed)


def chung_lu_induced(n: int, gamma: float, max_weight: float, mean_degree: float, seed: int, subset) -> Graph:
    """The subgraph of ``chung_lu(n, gamma, max_weight, mean_degree, seed)`` induced on ``subset``
    (distinct vertex ids), renumbered by the position of each vertex in the sorted subset.  Exactly
    the edges of the full graph between subset vertices: every row of the full graph has its own
    random stream, so only the subset's rows are drawn."""
    sub_ids = np.unique(np.asarray(subset, dtype=np.int64)).astype(np.int32)
    k = int(sub_ids.size)
    c, i0 = _chung_lu_scale(n, gamma, max_weight, mean_degree)
    name = f"chung_lu(n={n},gamma={gamma},seed={seed})[induced on {k} vertices]"
    if k == 0:
        return Graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32), name)
    import threading
    parts = max(1, min(64, (os.cpu_count() or 4) * 2, k))
    cuts = [k * j // parts for j in range(parts + 1)]
    out = [None] * parts
    psub = sub_ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    frac = k / max(n, 1)

    def work(j):
        a, b = cuts[j], cuts[j + 1]
        cap = int((b - a) * mean_degree * frac * 2) + 1024
        out[j] = _call_growing(_load().gg_chung_lu_induced, (n, gamma, c, i0, seed, psub, k, a, b), cap)

    th = [threading.Thread(target=work, args=(j,)) for j in range(parts)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return Graph(k, np.concatenate([o[0] for o in out]), np.concatenate([o[1] for o in out]), name)


def uniform_subset(n: int, k: int, seed: int) -> np.ndarray:
    """A seeded uniform k-subset of [0, n) (sorted int32): the first k of a SplitMix64-keyed
    permutation, i.e. the k vertices with the smallest hash of (seed, vertex)."""
    keys = np.empty(n, np.uint64)
    # vectorised SplitMix64 finaliser of (seed, v): the same stream definition as the C generators use
    z = np.arange(n, dtype=np.uint64) + np.uint64((seed * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    keys[:] = z ^ (z >> np.uint64(31))
    idx = np.argpartition(keys, k - 1)[:k] if 0 < k < n else np.arange(min(k, n))
    return np.sort(idx).astype(np.int32)


def chung_lu_large_induced(n_sub: int = 1_000_000, n_full: int = 50_000_000, seed: int = 1,
                           subset_seed: int = 2) -> Graph:
    """The partitioned large-graph workload's oracle check input: the subgraph of
    ``chung_lu_large(n_full, seed)`` induced on a seeded uniform n_sub-vertex subset."""
    sub_ids = uniform_subset(n_full, n_sub, subset_seed)
    return chung_lu_induced(n_full, 2.1, 1e6 * n_full / 50_000_000, 48.0, seed, sub_ids)


def batch_spec(seed: int, n_lo: int = 50, n_hi: int = 20000) -> BatchSpec:
    """Batched workload member ``seed``: generator uniform over {ER, BA, RGG}; n log-uniform in
    [n_lo, n_hi]; mean degree uniform in [4, 32] (ER, RGG); BA uses m uniform in {2..8}."""
    draw = [splitmix64_at(seed, 99, i) for i in range(4)]
    kind = ("er", "ba", "rgg")[draw[0] % 3]
    u = (draw[1] >> 11) * (1.0 / 9007199254740992.0)
    n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
    k = 4.0 + 28.0 * ((draw[2] >> 11) * (1.0 / 9007199254740992.0))
    m = 2 + int(draw[3] % 7)
    return BatchSpec(seed, kind, n, k, m)


def batch_graph(seed: int, n_lo: int = 50, n_hi: int = 20000) -> Graph:
    s = batch_spec(seed, n_lo, n_hi)
    if s.kind == "er":
        return er(s.n, s.k, 1000003 * seed + 17)
    if s.kind == "ba":
        return ba(s.n, min(s.m, max(1, s.n - 1)), 1000003 * seed + 17)
    return rgg(s.n, s.k, 1000003 * seed + 17)


@dataclass
class ServeSpec:
    seed: int
    kind: str       # "er" | "ba" | "rgg" | "rmat"
    m: int          # target edge count
    n: int
    k: float        # mean degree (er, rgg)
    attach: int     # edges per new vertex (ba)
    scale: int      # R-MAT scale (edge factor 16)


def serve_spec(seed: int, m_lo: float = 1e3, m_hi: float = 1e7) -> ServeSpec:
    """Served request ``seed``: target edge count log-uniform in [m_lo, m_hi]; generator uniform over
    {ER, BA, RGG, R-MAT (0.57, 0.19, 0.19)}; mean degree uniform in [4, 32] (ER, RGG), BA attaches
    m uniform in {2..8}, R-MAT uses edge factor 16 and the scale nearest the target."""
    draw = [splitmix64_at(seed, 77, i) for i in range(4)]
    kind = ("er", "ba", "rgg", "rmat")[draw[0] % 4]
    u = (draw[1] >> 11) * (1.0 / 9007199254740992.0)
    m = int(round(math.exp(math.log(m_lo) + u * (math.log(m_hi) - math.log(m_lo)))))
    k = 4.0 + 28.0 * ((draw[2] >> 11) * (1.0 / 9007199254740992.0))
    attach = 2 + int(draw[3] % 7)
    if kind == "ba":
        n = max(attach + 2, m // attach)
    else:
        n = max(8, int(round(2 * m / k)))
    scale = max(4, int(round(math.log2(max(m, 16) / 16))))
    return ServeSpec(seed, kind, m, n, k, attach, scale)


def serve_graph(seed: int, m_lo: float = 1e3, m_hi: float = 1e7) -> Graph:
    s = serve_spec(seed, m_lo, m_hi)
    gseed = 7919 * seed + 3
    if s.kind == "er":
        return er(s.n, s.k, gseed)
    if s.kind == "ba":
        return ba(s.n, s.attach, gseed)
    if s.kind == "rgg":
        return rgg(s.n, s.k, gseed)
    return rmat(s.scale, 16, 0.57, 0.19, 0.19, seed=gseed)
