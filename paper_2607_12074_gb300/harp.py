"""Thin ctypes binding of libharp (include/harp.h).  Argument marshalling only: every step of the
counting path runs in the library's CUDA kernels.  PyTorch tensors are accepted for device memory
(their data pointers are passed through) and torch streams for ordering.

The functions keep the C names (``harp_build_csr``, ``harp_count4`` ...).  There is no CPU fallback:
if libharp.so is missing or cannot be loaded, every call raises :class:`HarpUnavailable`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libharp.so")

HARP_OK, HARP_EINVAL, HARP_ENOMEM, HARP_ECUDA, HARP_EOVERFLOW = 0, 1, 2, 3, 4
HARP_EAGAIN, HARP_ETIMEOUT, HARP_ENOTFOUND, HARP_EDEVICE = 5, 6, 7, 8
HARP_PTR_HOST, HARP_PTR_DEVICE = 0, 1
HARP_ABI_VERSION = 2
HARP_BASIS_TRIANGLE_WEDGE, HARP_BASIS_LITERAL = 0, 1
HARP_PROBE_HASH, HARP_PROBE_BSEARCH = 1, 2
HARP_PLAN_NO_GRAPH, HARP_PLAN_NO_REUSE, HARP_PLAN_NO_BAND_MERGE = 1, 2, 4
HARP_NSEGMENTS = 9

MOTIFS = ("star3", "path4", "paw", "cycle4", "diamond", "clique4")
ORBITS = ("star_center", "star_leaf", "path_end", "path_inner", "paw_pendant", "paw_hub", "paw_side", "cycle",
          "diamond_spine", "diamond_tip", "clique")
HARP_NORBITS = 11
EDGE_ORBITS = ("star_edge", "path_end_edge", "path_mid_edge", "paw_pendant_edge", "paw_hub_edge",
               "paw_far_edge", "cycle_edge", "diamond_spine_edge", "diamond_rim_edge", "clique_edge")
HARP_NEDGE_ORBITS = 10
HARP_NMOTIFS5 = 21
STATS = ("T", "K4", "C4_non", "S_non", "P_non", "paw_non", "D_non", "m")


class HarpUnavailable(RuntimeError):
    """libharp.so is not built or cannot be loaded (no silent fallback exists)."""


class HarpError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {detail or status}")


class harp_plan(ctypes.Structure):
    _fields_ = [
        ("version", ctypes.c_uint32),
        ("basis", ctypes.c_uint32),
        ("tri_probe", ctypes.c_uint32),
        ("tri_warp_max", ctypes.c_uint32),
        ("tri_cta_max", ctypes.c_uint32),
        ("tri_big_max", ctypes.c_uint32),
        ("c4_warp_max_work", ctypes.c_uint32),
        ("c4_cta_max_work", ctypes.c_uint32),
        ("c4_window_bytes", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("est_enum", ctypes.c_double),
        ("est_inter", ctypes.c_double),
        ("est_halo", ctypes.c_double),
        ("est_reuse", ctypes.c_double),
        ("est_yield", ctypes.c_double),
        ("objective", ctypes.c_double),
        ("lit_cache_log2", ctypes.c_uint32),
        ("lit_cache_min_deg", ctypes.c_uint32),
        ("tri_probe_bin", ctypes.c_uint8 * 4),
        ("reserved0", ctypes.c_uint32),
        ("est_cost_tw", ctypes.c_double),
        ("est_cost_lit", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: (list(getattr(self, f)) if f == "tri_probe_bin" else getattr(self, f)) for f, _ in self._fields_}


class harp_select_opts(ctypes.Structure):
    _fields_ = [
        ("sample_vertices", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
        ("memory_budget", ctypes.c_uint64),
        ("lambda_inter", ctypes.c_double),
        ("lambda_halo", ctypes.c_double),
        ("lambda_reuse", ctypes.c_double),
        ("lambda_yield", ctypes.c_double),
    ]


class harp_partition_stats(ctypes.Structure):
    _fields_ = [("partitions", ctypes.c_int64), ("m", ctypes.c_int64), ("halo_arcs", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_uint64), ("device_peak_bytes", ctypes.c_uint64), ("host_ms", ctypes.c_double),
                ("transfer_ms", ctypes.c_double), ("device_ms", ctypes.c_double), ("graph_ms", ctypes.c_double),
                ("cut_ms", ctypes.c_double), ("tri_ms", ctypes.c_double), ("wedge_ms", ctypes.c_double),
                ("tri_blocks", ctypes.c_int64), ("wedge_blocks", ctypes.c_int64), ("wedge_sliced", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class harp_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("batch_window_us", ctypes.c_uint32), ("staging_mib", ctypes.c_uint32),
                ("small_edges", ctypes.c_uint32)]


class harp_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("completed", "batches", "batched_requests", "partitioned",
                                                "max_batch", "pending", "resident_bytes", "peak_resident_bytes",
                                                "latency_p50_us", "latency_p99_us")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def lib():
    """Load libharp.so (raises HarpUnavailable if absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise HarpUnavailable(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
        try:
            L = ctypes.CDLL(LIB_PATH)
        except OSError as e:
            raise HarpUnavailable(f"cannot load {LIB_PATH}: {e}") from e
        vp, i64, u32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
        pu64 = ctypes.POINTER(ctypes.c_uint64)
        pi64 = ctypes.POINTER(ctypes.c_int64)
        L.harp_build_csr.argtypes = [i64, i64, vp, vp, u32, vp, ctypes.POINTER(vp)]
        L.harp_csr_free.argtypes = [vp]
        L.harp_csr_free.restype = None
        L.harp_csr_info.argtypes = [vp, pi64, pi64, pi64, ctypes.POINTER(ctypes.c_size_t)]
        L.harp_csr_arrays.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.harp_select_anchors.argtypes = [vp, ctypes.POINTER(harp_select_opts), ctypes.POINTER(harp_plan)]
        L.harp_count4.argtypes = [vp, ctypes.POINTER(harp_plan), pu64]
        L.harp_count4_stats.argtypes = [vp, ctypes.POINTER(harp_plan), pu64, pu64]
        L.harp_reuse_stats.argtypes = [vp, pu64, pu64]
        L.harp_reuse_stats.restype = i32
        L.harp_count4_async.argtypes = [vp, ctypes.POINTER(harp_plan), vp, vp]
        L.harp_count4_noalloc.argtypes = [i64, i64, vp, vp, vp, vp]
        L.harp_count4_orbits.argtypes = [vp, vp, u32]
        L.harp_count4_orbits.restype = i32
        L.harp_count4_edge_orbits.argtypes = [vp, vp, u32]
        L.harp_count4_edge_orbits.restype = i32
        L.harp_count5.argtypes = [vp, pu64]
        L.harp_count5.restype = i32
        L.harp_motif5_classes.argtypes = [ctypes.POINTER(ctypes.c_uint16)]
        L.harp_motif5_classes.restype = i32
        L.harp_batch_create.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(vp)]
        L.harp_batch_count.argtypes = [vp, ctypes.POINTER(harp_plan), vp, vp, vp]
        L.harp_batch_info.argtypes = [vp, pi64, pi64, pi64, ctypes.POINTER(ctypes.c_size_t)]
        L.harp_batch_free.argtypes = [vp]
        L.harp_batch_free.restype = None
        L.harp_count4_batch.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(harp_plan), vp, vp]
        L.harp_batch_autotune.argtypes = [vp, ctypes.POINTER(harp_plan), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(harp_plan), ctypes.POINTER(ctypes.c_float)]
        for name in ("harp_batch_create", "harp_batch_count", "harp_batch_info", "harp_count4_batch",
                     "harp_batch_autotune"):
            getattr(L, name).restype = i32
        L.harp_count4_partitioned.argtypes = [i64, i64, vp, vp, ctypes.c_uint64, ctypes.c_int32, pu64,
                                              ctypes.POINTER(harp_partition_stats)]
        L.harp_partition_plan.argtypes = [i64, i64, vp, vp, ctypes.c_uint64, ctypes.c_int32,
                                          ctypes.POINTER(harp_partition_stats), pi64, pi64, i64]
        L.harp_rank_csr_host.argtypes = [i64, i64, vp, vp, pi64, ctypes.POINTER(ctypes.c_int32), pi64,
                                         ctypes.POINTER(ctypes.c_int32), i64]
        L.harp_server_create.argtypes = [ctypes.POINTER(harp_server_opts), ctypes.POINTER(vp)]
        L.harp_submit.argtypes = [vp, i64, i64, vp, vp, pu64]
        L.harp_poll.argtypes = [vp, ctypes.c_uint64, pu64, ctypes.POINTER(ctypes.c_int)]
        L.harp_wait.argtypes = [vp, ctypes.c_uint64, pu64, ctypes.c_double]
        L.harp_server_get_stats.argtypes = [vp, ctypes.POINTER(harp_server_stats)]
        L.harp_server_destroy.argtypes = [vp]
        L.harp_server_destroy.restype = None
        for name in ("harp_count4_partitioned", "harp_partition_plan", "harp_rank_csr_host", "harp_server_create", "harp_submit", "harp_poll", "harp_wait",
                     "harp_server_get_stats"):
            getattr(L, name).restype = i32
        L.harp_set_profiling.argtypes = [i32]
        L.harp_last_stage_times.argtypes = [ctypes.POINTER(ctypes.c_float), pi64]
        L.harp_launch_count.argtypes = []
        L.harp_launch_count.restype = i64
        L.harp_status_str.argtypes = [i32]
        L.harp_status_str.restype = ctypes.c_char_p
        L.harp_last_cuda_error.argtypes = []
        L.harp_last_cuda_error.restype = i32
        L.harp_last_cuda_error_str.argtypes = []
        L.harp_last_cuda_error_str.restype = ctypes.c_char_p
        for name in ("harp_build_csr", "harp_csr_info", "harp_csr_arrays", "harp_select_anchors", "harp_count4",
                     "harp_count4_stats", "harp_count4_async", "harp_count4_noalloc", "harp_set_profiling",
                     "harp_last_stage_times"):
            getattr(L, name).restype = i32
        _lib = L
        return L


def _check(st: int, what: str):
    if st != HARP_OK:
        L = lib()
        detail = L.harp_status_str(st).decode()
        if st == HARP_ECUDA:
            detail += f" ({L.harp_last_cuda_error_str().decode()})"
        raise HarpError(st, what, detail)


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _edge_ptrs(src, dst):
    """Return (ptr_src, ptr_dst, m_in, flags, keepalive)."""
    try:
        import torch
        if isinstance(src, torch.Tensor):
            if not (src.is_cuda and dst.is_cuda):
                src, dst = src.cpu().numpy(), dst.cpu().numpy()
            else:
                if src.dtype != torch.int32 or dst.dtype != torch.int32:
                    raise TypeError("device edge lists must be torch.int32")
                src, dst = src.contiguous(), dst.contiguous()
                if src.numel() != dst.numel():
                    raise ValueError("src and dst differ in length")
                return src.data_ptr(), dst.data_ptr(), src.numel(), HARP_PTR_DEVICE, (src, dst)
    except ImportError:
        pass
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    if s.shape != d.shape or s.ndim != 1:
        raise ValueError("src and dst must be 1-D and of equal length")
    return s.ctypes.data, d.ctypes.data, s.size, HARP_PTR_HOST, (s, d)


class Csr:
    """Owns a harp_csr handle (device memory); freed on close() or garbage collection."""

    def __init__(self, handle: int, keepalive=None):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keepalive

    def close(self):
        if self.handle:
            lib().harp_csr_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return harp_csr_info(self)


def harp_build_csr(n: int, src, dst, stream=None) -> Csr:
    """Device CSR from an undirected edge list (numpy/host arrays or torch.int32 CUDA tensors)."""
    ps, pd, m_in, flags, keep = _edge_ptrs(src, dst)
    out = ctypes.c_void_p()
    st = lib().harp_build_csr(int(n), int(m_in), ps, pd, flags, _stream_handle(stream), ctypes.byref(out))
    _check(st, "harp_build_csr")
    return Csr(out.value, None)


def harp_csr_info(g: Csr) -> dict:
    n, m, md = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    b = ctypes.c_size_t()
    _check(lib().harp_csr_info(g.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(md), ctypes.byref(b)),
           "harp_csr_info")
    return {"n": n.value, "m": m.value, "max_degree": md.value, "device_bytes": b.value}


def harp_csr_arrays(g: Csr) -> tuple[int, int]:
    off, cols = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().harp_csr_arrays(g.handle, ctypes.byref(off), ctypes.byref(cols)), "harp_csr_arrays")
    return off.value, cols.value


def harp_select_anchors(g: Csr, sample_vertices: int = 0, seed: int = 0, memory_budget: int = 0) -> harp_plan:
    """The Eq. 1 plan for g: the cheaper of the two bases (plan.basis), both objectives in
    est_cost_tw / est_cost_lit."""
    opts = harp_select_opts(sample_vertices, seed, memory_budget, 0.0, 0.0, 0.0, 0.0)
    p = harp_plan()
    p.version = HARP_ABI_VERSION
    _check(lib().harp_select_anchors(g.handle, ctypes.byref(opts), ctypes.byref(p)), "harp_select_anchors")
    return p


def _plan_ref(plan):
    return ctypes.byref(plan) if plan is not None else None


def harp_count4(g: Csr, plan: harp_plan | None = None) -> np.ndarray:
    """The six induced counts [star3, path4, paw, cycle4, diamond, clique4] as numpy uint64."""
    out = np.zeros(6, np.uint64)
    _check(lib().harp_count4(g.handle, _plan_ref(plan), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))),
           "harp_count4")
    return out


def harp_reuse_stats(g: Csr) -> tuple[int, int]:
    """(lookups, hits) of the signature reuse in the last blocking count on g."""
    lk, ht = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().harp_reuse_stats(g.handle, ctypes.byref(lk), ctypes.byref(ht)), "harp_reuse_stats")
    return lk.value, ht.value


def harp_count4_stats(g: Csr, plan: harp_plan | None = None) -> tuple[np.ndarray, np.ndarray]:
    out = np.zeros(6, np.uint64)
    st = np.zeros(8, np.uint64)
    _check(lib().harp_count4_stats(g.handle, _plan_ref(plan), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "harp_count4_stats")
    return out, st


def harp_count4_async(g: Csr, d_out_ptr: int, plan: harp_plan | None = None, stream=None) -> None:
    """Enqueue a count; d_out_ptr is a device pointer to >= 16 uint64 (e.g. a torch int64 tensor)."""
    _check(lib().harp_count4_async(g.handle, _plan_ref(plan), ctypes.c_void_p(d_out_ptr), _stream_handle(stream)),
           "harp_count4_async")


def harp_count4_orbits(g: Csr, out=None) -> np.ndarray:
    """Per-vertex orbit counts uint64[n, 11] (rows = input vertex ids, columns in ORBITS order).
    out: None (a new host array) or a torch.int64 CUDA tensor of n * 11 elements (filled in place)."""
    n = g.info()["n"]
    if out is not None:
        _check(lib().harp_count4_orbits(g.handle, ctypes.c_void_p(out.data_ptr()), HARP_PTR_DEVICE),
               "harp_count4_orbits")
        return out
    res = np.zeros((n, HARP_NORBITS), np.uint64)
    _check(lib().harp_count4_orbits(g.handle, ctypes.c_void_p(res.ctypes.data if n else 0), HARP_PTR_HOST),
           "harp_count4_orbits")
    return res


def harp_count4_edge_orbits(g: Csr, out=None) -> np.ndarray:
    """Per-edge orbit counts uint64[m, 10] (rows = edges (a, b), a < b, in lexicographic order of the input
    ids; columns in EDGE_ORBITS order).  out: None (a new host array) or a torch.int64 CUDA tensor of
    m * 10 elements (filled in place)."""
    m = g.info()["m"]
    if out is not None:
        _check(lib().harp_count4_edge_orbits(g.handle, ctypes.c_void_p(out.data_ptr()), HARP_PTR_DEVICE),
               "harp_count4_edge_orbits")
        return out
    res = np.zeros((m, HARP_NEDGE_ORBITS), np.uint64)
    _check(lib().harp_count4_edge_orbits(g.handle, ctypes.c_void_p(res.ctypes.data if m else 0), HARP_PTR_HOST),
           "harp_count4_edge_orbits")
    return res


def harp_count5(g: Csr) -> np.ndarray:
    """Connected induced 5-vertex motif counts uint64[21], classes in harp_motif5_classes() order."""
    out = np.zeros(HARP_NMOTIFS5, np.uint64)
    _check(lib().harp_count5(g.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "harp_count5")
    return out


def harp_motif5_classes() -> list[int]:
    """The 21 class keys (10-bit canonical adjacency masks over the lexicographic vertex pairs) in order."""
    keys = (ctypes.c_uint16 * HARP_NMOTIFS5)()
    _check(lib().harp_motif5_classes(keys), "harp_motif5_classes")
    return list(keys)


def harp_count4_noalloc(n: int, m: int, d_offsets: int, d_cols: int, d_out: int, stream=None) -> None:
    """Count a device CSR (n <= 262,144, m <= 524,288) without any device allocation.

    For callers that may not allocate device memory while they run.  d_offsets / d_cols / d_out
    are device pointers (int64[n+1], int32[2m], uint64[16]); the work is only enqueued on `stream`.
    d_out[6] is the device self-check word (0 = fine; nonzero = a CSR whose sizes or ids failed the
    check, counted as edgeless).  Scratch is a static 64 MiB device array shared by all calls:
    serialise calls that could overlap.
    """
    _check(lib().harp_count4_noalloc(int(n), int(m), ctypes.c_void_p(d_offsets), ctypes.c_void_p(d_cols),
                                     ctypes.c_void_p(d_out), _stream_handle(stream)), "harp_count4_noalloc")


class Batch:
    """Owns a harp_batch (the packed union of many handles and its captured CUDA graph)."""

    def __init__(self, handle: int, G: int):
        self.handle = ctypes.c_void_p(handle)
        self.G = G

    def close(self):
        if self.handle:
            lib().harp_batch_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def harp_batch_create(graphs) -> Batch:
    arr = (ctypes.c_void_p * max(1, len(graphs)))(*[g.handle.value for g in graphs])
    out = ctypes.c_void_p()
    _check(lib().harp_batch_create(arr, len(graphs), ctypes.byref(out)), "harp_batch_create")
    return Batch(out.value, len(graphs))


def harp_batch_count(b: Batch, plan: harp_plan | None = None, stream=None, stats: bool = False):
    counts = np.zeros((max(1, b.G), 6), np.uint64)
    st = np.zeros((max(1, b.G), 8), np.uint64)
    _check(lib().harp_batch_count(b.handle, _plan_ref(plan), counts.ctypes.data, st.ctypes.data if stats else None,
                                  _stream_handle(stream)), "harp_batch_count")
    return (counts[:b.G], st[:b.G]) if stats else counts[:b.G]


def harp_batch_info(b: Batch) -> dict:
    g, n, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    by = ctypes.c_size_t()
    _check(lib().harp_batch_info(b.handle, ctypes.byref(g), ctypes.byref(n), ctypes.byref(m), ctypes.byref(by)),
           "harp_batch_info")
    return {"graphs": g.value, "n": n.value, "m": m.value, "device_bytes": by.value}


HARP_AUTOTUNE_GRID = 24


def harp_batch_autotune(b: Batch, candidates=None, reps: int = 3):
    """Time each candidate plan (default: the built-in grid) on the batch; returns (best plan, ms list)."""
    if candidates:
        arr = (harp_plan * len(candidates))(*candidates)
        nc = len(candidates)
    else:
        arr, nc = None, HARP_AUTOTUNE_GRID
    ms = (ctypes.c_float * nc)()
    best = harp_plan()
    _check(lib().harp_batch_autotune(b.handle, arr, nc if candidates else 0, int(reps), ctypes.byref(best), ms),
           "harp_batch_autotune")
    return best, [float(x) for x in ms]


def harp_count4_batch(graphs, plan: harp_plan | None = None, stream=None) -> np.ndarray:
    arr = (ctypes.c_void_p * max(1, len(graphs)))(*[g.handle.value for g in graphs])
    counts = np.zeros((max(1, len(graphs)), 6), np.uint64)
    _check(lib().harp_count4_batch(arr, len(graphs), _plan_ref(plan), counts.ctypes.data, _stream_handle(stream)),
           "harp_count4_batch")
    return counts[:len(graphs)]


def harp_count4_partitioned(n: int, src, dst, budget_bytes: int = 0, parts: int = 0):
    """Counts of a graph given as a host edge list, by owner-rule partitions under a device budget.

    Returns (counts uint64[6], stats dict)."""
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    out = np.zeros(6, np.uint64)
    st = harp_partition_stats()
    _check(lib().harp_count4_partitioned(int(n), s.size, s.ctypes.data, d.ctypes.data, int(budget_bytes), int(parts),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(st)),
           "harp_count4_partitioned")
    return out, st.as_dict()


def harp_partition_plan(n: int, src, dst, budget_bytes: int, parts: int = 0):
    """Host-only dry run of harp_count4_partitioned (no device work).

    Returns (stats dict, triangle ranges int64[k, 2], wedge blocks int64[w, 4]) in rank order."""
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    cap = 1024
    while True:
        st = harp_partition_stats()
        tri = np.zeros((cap, 2), np.int64)
        wedge = np.zeros((cap, 4), np.int64)
        _check(lib().harp_partition_plan(int(n), s.size, s.ctypes.data, d.ctypes.data, int(budget_bytes), int(parts),
                                         ctypes.byref(st), tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         wedge.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap),
               "harp_partition_plan")
        if st.tri_blocks <= cap and st.wedge_blocks <= cap:
            return st.as_dict(), tri[:st.tri_blocks].copy(), wedge[:st.wedge_blocks].copy()
        cap = max(st.tri_blocks, st.wedge_blocks)


def harp_rank_csr_host(n: int, src, dst):
    """The host rank-order graph of the partitioned path: (rank int32[n], offsets int64[n+1], cols int32[2m])."""
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    m = ctypes.c_int64()
    _check(lib().harp_rank_csr_host(int(n), s.size, s.ctypes.data, d.ctypes.data, ctypes.byref(m), None, None, None, 0),
           "harp_rank_csr_host")
    rank = np.zeros(n, np.int32)
    off = np.zeros(n + 1, np.int64)
    cols = np.zeros(max(2 * m.value, 1), np.int32)
    p32 = ctypes.POINTER(ctypes.c_int32)
    _check(lib().harp_rank_csr_host(int(n), s.size, s.ctypes.data, d.ctypes.data, ctypes.byref(m),
                                    rank.ctypes.data_as(p32), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    cols.ctypes.data_as(p32), cols.size), "harp_rank_csr_host")
    return rank, off, cols[:2 * m.value]


class Server:
    """A continuous-batching counting server (harp_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 0, max_batch: int = 0, max_inflight: int = 0,
                 batch_window_us: int = 0, staging_mib: int = 0, small_edges: int = 0):
        o = harp_server_opts(hbm_budget_bytes, max_batch, max_inflight, batch_window_us, staging_mib, small_edges)
        h = ctypes.c_void_p()
        _check(lib().harp_server_create(ctypes.byref(o), ctypes.byref(h)), "harp_server_create")
        self.handle = h

    def submit(self, n: int, src, dst) -> int:
        s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
        d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
        t = ctypes.c_uint64()
        _check(lib().harp_submit(self.handle, int(n), s.size, s.ctypes.data, d.ctypes.data, ctypes.byref(t)),
               "harp_submit")
        return t.value

    def poll(self, ticket: int):
        """None while running; the counts once done (raises HarpError on a failed request)."""
        out = np.zeros(6, np.uint64)
        done = ctypes.c_int(0)
        st = lib().harp_poll(self.handle, ticket, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                             ctypes.byref(done))
        _check(st, "harp_poll")
        return out if done.value else None

    def wait(self, ticket: int, timeout_ms: float = -1.0) -> np.ndarray:
        out = np.zeros(6, np.uint64)
        _check(lib().harp_wait(self.handle, ticket, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               float(timeout_ms)), "harp_wait")
        return out

    def stats(self) -> dict:
        st = harp_server_stats()
        _check(lib().harp_server_get_stats(self.handle, ctypes.byref(st)), "harp_server_get_stats")
        return st.as_dict()

    def close(self):
        if self.handle:
            lib().harp_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def harp_set_profiling(enable: bool) -> None:
    _check(lib().harp_set_profiling(1 if enable else 0), "harp_set_profiling")


def harp_last_stage_times() -> tuple[list[float], int]:
    ms = (ctypes.c_float * HARP_NSEGMENTS)()
    launches = ctypes.c_int64()
    _check(lib().harp_last_stage_times(ms, ctypes.byref(launches)), "harp_last_stage_times")
    return list(ms), launches.value


def harp_launch_count() -> int:
    return int(lib().harp_launch_count())


def count4_edges(n: int, src, dst, plan: harp_plan | None = None, stream=None) -> np.ndarray:
    """Convenience: build the CSR from an edge list, count, free."""
    g = harp_build_csr(n, src, dst, stream)
    try:
        return harp_count4(g, plan)
    finally:
        g.close()
