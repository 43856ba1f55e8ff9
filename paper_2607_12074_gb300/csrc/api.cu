// The C ABI of libharp (include/harp.h): argument checking, handles, workspaces and the counting
// pipeline a1 -> a3/a4 -> a5 -> a7 on one stream.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>

#include "harp_internal.cuh"

namespace harp {

namespace {
thread_local cudaError_t t_last_err = cudaSuccess;
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_profiling{0};
float g_stage_ms[HARP_NSEGMENTS] = {0};
int64_t g_stage_launches = 0;
// events of the count being profiled: [0] start, [1 + seg] end of segment seg
thread_local cudaEvent_t t_marks[HARP_NSEGMENTS + 1] = {nullptr};
thread_local bool t_marked[HARP_NSEGMENTS + 1] = {false};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

void record_cuda_error(cudaError_t e) {
    if (t_last_err == cudaSuccess) t_last_err = e;
}
void note_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int num_sms() {
    static std::atomic<int> cached[64];  // 0 = not queried yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 152;
    cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

cudaError_t prof_mark(cudaStream_t s, int seg) {
    if (!g_profiling.load(std::memory_order_relaxed) || !t_marks[0]) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return cudaSuccess;
    t_marked[seg + 1] = true;
    return cudaEventRecord(t_marks[seg + 1], s);
}

size_t ws_layout(Workspace& ws, unsigned char* base, int64_t n, int64_t m) {
    const int64_t nn = n > 0 ? n : 1;
    const int64_t mm = m > 0 ? m : 1;
    const size_t hist_len = radix_hist_len(nn);
    const size_t tmp_len = scan_tmp_needed(nn) + scan_tmp_needed((int64_t)hist_len) + 64;
    struct Part { void** p; size_t bytes; };
    Part parts[] = {
        {(void**)&ws.deg, sizeof(int32_t) * nn},
        {(void**)&ws.order, sizeof(int32_t) * nn},
        {(void**)&ws.perm, sizeof(int32_t) * nn},
        {(void**)&ws.dplus, sizeof(int32_t) * nn},
        {(void**)&ws.fpos, sizeof(int32_t) * nn},
        {(void**)&ws.rev, sizeof(int32_t) * 2 * mm},
        {(void**)&ws.bpos, sizeof(int32_t) * kGridCap * nn},
        {(void**)&ws.ginfo, sizeof(int64_t) * kGInfo},
        {(void**)&ws.vkeys, sizeof(uint64_t) * nn},
        {(void**)&ws.vkeys_alt, sizeof(uint64_t) * nn},
        {(void**)&ws.hist, sizeof(uint32_t) * hist_len},
        {(void**)&ws.off, sizeof(int64_t) * (nn + 1)},
        {(void**)&ws.offp, sizeof(int64_t) * (nn + 1)},
        {(void**)&ws.cols, sizeof(int32_t) * 2 * mm},
        {(void**)&ws.colsp, sizeof(int32_t) * 2 * mm},  // colsp [m] followed by te [m]
        {(void**)&ws.q_tri, sizeof(int32_t) * nn},
        {(void**)&ws.q_mid, sizeof(int32_t) * 2 * nn},
        {(void**)&ws.q_win, sizeof(int32_t) * 2 * nn},
        {(void**)&ws.win_prefix, sizeof(int64_t) * (nn + 1)},
        {(void**)&ws.scan_tmp, sizeof(int64_t) * tmp_len},
        {(void**)&ws.acc, sizeof(uint64_t) * kOutLen},
    };
    size_t total = 0;
    for (const Part& p : parts) {
        if (base) *p.p = base + total;
        total += align_up(p.bytes);
    }
    if (base) {
        ws.te = reinterpret_cast<uint32_t*>(ws.colsp + mm);
        ws.hist_len = hist_len;
        ws.scan_tmp_len = tmp_len;
        ws.base = base;
        ws.bytes = total;
        ws.n = n;
        ws.m = m;
    }
    return total;
}

harp_status ws_ensure(Workspace& ws, int64_t n, int64_t m, cudaStream_t s) {
    if (ws.base && ws.n == n && ws.m == m) return HARP_OK;
    ws_release(ws, s);
    Workspace probe;
    const size_t total = ws_layout(probe, nullptr, n, m);
    void* base = nullptr;
    cudaError_t e = cudaMallocAsync(&base, total, s);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
    }
    ws_layout(ws, static_cast<unsigned char*>(base), n, m);
    return HARP_OK;
}

// The stream-ordered allocator's default pool keeps freed memory for reuse (no release back to the
// driver at synchronisation), so repeated builds and counts do not pay for fresh allocations.
void ensure_pool(int device) {
    static std::atomic<uint64_t> done{0};
    const uint64_t bit = device < 64 ? (1ull << device) : 0;
    if (!bit || (done.load() & bit)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done.fetch_or(bit);
}

void ws_release(Workspace& ws, cudaStream_t s) {
    if (ws.base) cudaFreeAsync(ws.base, s);
    ws = Workspace();
}

namespace {

harp_status validate_plan(const harp_plan* p) {
    if (!p) return HARP_OK;
    if (p->version != 0 && p->version != 1 && p->version != HARP_ABI_VERSION) return HARP_EINVAL;
    if (p->basis != HARP_BASIS_TRIANGLE_WEDGE && p->basis != HARP_BASIS_LITERAL) return HARP_EINVAL;
    return HARP_OK;
}

// The whole count enqueued on stream s; results land in ws.acc.
harp_status enqueue_count(harp_csr* g, const harp_plan* user_plan, cudaStream_t s) {
    HARP_TRY(validate_plan(user_plan));
    harp_plan plan;
    normalise_plan(user_plan, &plan);
    HARP_TRY(ws_ensure(g->ws, g->n, g->m, s));
    Workspace& ws = g->ws;
    HARP_CK(cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s));
    const bool prof = g_profiling.load() != 0;
    if (prof) {
        for (int k = 0; k <= HARP_NSEGMENTS; ++k) {
            if (!t_marks[k]) HARP_CK(cudaEventCreate(&t_marks[k]));
            t_marked[k] = false;
        }
        HARP_CK(cudaEventRecord(t_marks[0], s));
        t_marked[0] = true;
    }
    const int64_t l0 = g_launches.load();
    harp_status st = orient(g, ws, s);
    if (st == HARP_OK) st = prof_mark(s, SEG_ORIENT) == cudaSuccess ? HARP_OK : HARP_ECUDA;
    if (plan.basis == HARP_BASIS_LITERAL) {
        if (st == HARP_OK) st = count_literal(g, ws, plan, s);
    } else {
        if (st == HARP_OK) st = count_triangles_k4(g, ws, plan, s);
        if (st == HARP_OK) st = count_wedge_c4(g, ws, plan, s);
        if (st == HARP_OK) st = reduce_and_close(g, ws, s);
    }
    if (st == HARP_OK) st = prof_mark(s, SEG_REDUCE) == cudaSuccess ? HARP_OK : HARP_ECUDA;
    if (prof && st == HARP_OK && cudaEventSynchronize(t_marks[HARP_NSEGMENTS]) == cudaSuccess) {
        int prev = 0;
        for (int k = 1; k <= HARP_NSEGMENTS; ++k) {
            g_stage_ms[k - 1] = 0.0f;
            if (!t_marked[k]) continue;
            cudaEventElapsedTime(&g_stage_ms[k - 1], t_marks[prev], t_marks[k]);
            prev = k;
        }
        g_stage_launches = g_launches.load() - l0;
    }
    if (prof) {
        for (int k = 0; k <= HARP_NSEGMENTS; ++k) t_marked[k] = false;
    }
    return st;
}

harp_status count_to_host(const harp_csr* gc, const harp_plan* plan, uint64_t* counts_out, uint64_t* stats_out) {
    if (!gc || !counts_out) return HARP_EINVAL;
    harp_csr* g = const_cast<harp_csr*>(gc);
    HARP_CK(cudaSetDevice(g->device));
    HARP_TRY(enqueue_count(g, plan, g->stream));
    uint64_t host[kOutLen];
    HARP_CK(cudaMemcpyAsync(host, g->ws.acc, sizeof(host), cudaMemcpyDeviceToHost, g->stream));
    HARP_CK(cudaStreamSynchronize(g->stream));
    if (host[ACC_ERR]) return HARP_EDEVICE;  // a kernel's self-check skipped an out-of-range access
    const bool literal = plan && plan->basis == HARP_BASIS_LITERAL;
    g->sig_lookups = literal ? host[ACC_SIG_LOOKUPS] : host[ACC_T];
    g->sig_hits = host[ACC_SIG_HITS];
    g->have_reuse = true;
    std::memcpy(counts_out, host + OUT_COUNTS, 6 * sizeof(uint64_t));
    if (stats_out) std::memcpy(stats_out, host + OUT_STATS, HARP_NSTATS * sizeof(uint64_t));
    return HARP_OK;
}

}  // namespace
}  // namespace harp

namespace harp {
namespace {
// shared body of the per-vertex and per-edge orbit outputs: orientation, the triangle pass (t_e of
// every out-arc), then `run` writes rows*cols uint64 into the device output
template <typename Run>
harp_status orbit_output(harp_csr* g, uint64_t* orbits_out, uint32_t flags, size_t rows, size_t cols, Run run) {
    cudaStream_t s = g->stream;
    HARP_TRY(ws_ensure(g->ws, g->n, g->m, s));
    Workspace& ws = g->ws;
    HARP_CK(cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s));
    harp_plan plan;
    normalise_plan(nullptr, &plan);
    const size_t out_bytes = sizeof(uint64_t) * cols * rows;
    uint64_t* d_out = orbits_out;
    if (flags == HARP_PTR_HOST) HARP_CK(cudaMallocAsync((void**)&d_out, out_bytes, s));
    harp_status st = orient(g, ws, s);
    if (st == HARP_OK) st = count_triangles_k4(g, ws, plan, s);
    if (st == HARP_OK) st = run(ws, d_out, s);
    uint64_t err = 0;
    cudaError_t e = cudaSuccess;
    if (st == HARP_OK) e = cudaMemcpyAsync(&err, ws.acc + ACC_ERR, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (st == HARP_OK && e == cudaSuccess && flags == HARP_PTR_HOST)
        e = cudaMemcpyAsync(orbits_out, d_out, out_bytes, cudaMemcpyDeviceToHost, s);
    if (flags == HARP_PTR_HOST) cudaFreeAsync(d_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return HARP_ECUDA;
    }
    if (st != HARP_OK) return st;
    return err ? HARP_EDEVICE : HARP_OK;
}
}  // namespace
}  // namespace harp

using namespace harp;

extern "C" {

harp_status harp_build_csr(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, uint32_t flags,
                           void* stream, harp_csr** out) {
    if (!out) return HARP_EINVAL;
    if (n < 0 || m_in < 0) return HARP_EINVAL;
    if (n > 2147483647LL || m_in > 2147483647LL) return HARP_EOVERFLOW;
    if (m_in > 0 && (!src || !dst)) return HARP_EINVAL;
    if (flags != HARP_PTR_HOST && flags != HARP_PTR_DEVICE) return HARP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    harp_csr* g = new (std::nothrow) harp_csr();
    if (!g) return HARP_ENOMEM;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return HARP_ECUDA;
    }
    ensure_pool(g->device);
    g->stream = s;
    const int32_t* d_src = src;
    const int32_t* d_dst = dst;
    int32_t* staged = nullptr;
    harp_status st = HARP_OK;
    if (flags == HARP_PTR_HOST && m_in > 0) {
        cudaError_t e = cudaMallocAsync((void**)&staged, 2 * (size_t)m_in * sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(staged, src, (size_t)m_in * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(staged + m_in, dst, (size_t)m_in * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            st = e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
        }
        d_src = staged;
        d_dst = staged + m_in;
    }
    if (st == HARP_OK) st = build_csr_device(g, n, m_in, d_src, d_dst, s);
    if (staged) cudaFreeAsync(staged, s);
    if (st != HARP_OK) {
        if (g->off) cudaFreeAsync(g->off, s);
        if (g->cols) cudaFreeAsync(g->cols, s);
        cudaStreamSynchronize(s);
        delete g;
        return st;
    }
    *out = g;
    return HARP_OK;
}

harp_status harp_reuse_stats(const harp_csr* g, uint64_t* lookups, uint64_t* hits) {
    if (!g) return HARP_EINVAL;
    if (!g->have_reuse) return HARP_ENOTFOUND;
    if (lookups) *lookups = g->sig_lookups;
    if (hits) *hits = g->sig_hits;
    return HARP_OK;
}

void harp_csr_free(harp_csr* g) {
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    // stream-ordered frees: they run after the work already queued on the handle's stream, and the
    // caller is not blocked (a server frees handles while other streams keep working)
    ws_release(g->ws, g->stream);
    if (g->off) cudaFreeAsync(g->off, g->stream);
    if (g->cols) cudaFreeAsync(g->cols, g->stream);
    cudaSetDevice(prev);
    delete g;
}

harp_status harp_csr_info(const harp_csr* g, int64_t* n, int64_t* m_undirected, int64_t* max_degree,
                          size_t* device_bytes) {
    if (!g) return HARP_EINVAL;
    if (n) *n = g->n;
    if (m_undirected) *m_undirected = g->m;
    if (max_degree) *max_degree = g->max_deg;
    if (device_bytes) *device_bytes = g->csr_bytes + g->ws.bytes;
    return HARP_OK;
}

harp_status harp_csr_arrays(const harp_csr* g, const int64_t** offsets, const int32_t** cols) {
    if (!g || !offsets || !cols) return HARP_EINVAL;
    *offsets = g->off;
    *cols = g->cols;
    return HARP_OK;
}

harp_status harp_count4(const harp_csr* g, const harp_plan* plan, uint64_t counts_out[6]) {
    return count_to_host(g, plan, counts_out, nullptr);
}

harp_status harp_count4_stats(const harp_csr* g, const harp_plan* plan, uint64_t counts_out[6],
                              uint64_t stats_out[8]) {
    if (!stats_out) return HARP_EINVAL;
    return count_to_host(g, plan, counts_out, stats_out);
}

harp_status harp_count4_async(const harp_csr* gc, const harp_plan* plan, uint64_t* d_out, void* stream) {
    if (!gc || !d_out) return HARP_EINVAL;
    harp_csr* g = const_cast<harp_csr*>(gc);
    cudaStream_t s = (cudaStream_t)stream;
    HARP_CK(cudaSetDevice(g->device));
    HARP_TRY(enqueue_count(g, plan, s));
    HARP_CK(cudaMemcpyAsync(d_out, g->ws.acc, 16 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    HARP_CK(cudaMemcpyAsync(d_out + OUT_ERR, g->ws.acc + ACC_ERR, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return HARP_OK;
}

harp_status harp_count4_edge_orbits(const harp_csr* gc, uint64_t* orbits_out, uint32_t flags) {
    if (!gc || (!orbits_out && gc->m > 0)) return HARP_EINVAL;
    if (flags != HARP_PTR_HOST && flags != HARP_PTR_DEVICE) return HARP_EINVAL;
    harp_csr* g = const_cast<harp_csr*>(gc);
    if (g->m == 0) return HARP_OK;
    HARP_CK(cudaSetDevice(g->device));
    return orbit_output(g, orbits_out, flags, (size_t)g->m, HARP_NEDGE_ORBITS,
                        [&](Workspace& ws, uint64_t* d_out, cudaStream_t s) { return count_edge_orbits(g, ws, d_out, s); });
}

harp_status harp_count4_orbits(const harp_csr* gc, uint64_t* orbits_out, uint32_t flags) {
    if (!gc || (!orbits_out && gc->n > 0)) return HARP_EINVAL;
    if (flags != HARP_PTR_HOST && flags != HARP_PTR_DEVICE) return HARP_EINVAL;
    harp_csr* g = const_cast<harp_csr*>(gc);
    if (g->n == 0) return HARP_OK;
    HARP_CK(cudaSetDevice(g->device));
    return orbit_output(g, orbits_out, flags, (size_t)g->n, HARP_NORBITS,
                        [&](Workspace& ws, uint64_t* d_out, cudaStream_t s) { return count_orbits(g, ws, d_out, s); });
}

harp_status harp_set_profiling(int enable) {
    g_profiling.store(enable ? 1 : 0);
    return HARP_OK;
}

harp_status harp_last_stage_times(float ms_out[HARP_NSEGMENTS], int64_t* launches_out) {
    if (!ms_out) return HARP_EINVAL;
    for (int k = 0; k < HARP_NSEGMENTS; ++k) ms_out[k] = g_stage_ms[k];
    if (launches_out) *launches_out = g_stage_launches;
    return HARP_OK;
}

int64_t harp_launch_count(void) { return g_launches.load(); }

const char* harp_status_str(harp_status s) {
    switch (s) {
        case HARP_OK: return "HARP_OK";
        case HARP_EINVAL: return "HARP_EINVAL: invalid argument";
        case HARP_ENOMEM: return "HARP_ENOMEM: out of memory or over budget";
        case HARP_ECUDA: return "HARP_ECUDA: CUDA runtime error";
        case HARP_EOVERFLOW: return "HARP_EOVERFLOW: size exceeds the index types";
        case HARP_EAGAIN: return "HARP_EAGAIN: not finished";
        case HARP_ETIMEOUT: return "HARP_ETIMEOUT: bounded device wait expired";
        case HARP_ENOTFOUND: return "HARP_ENOTFOUND: unknown ticket or handle";
        case HARP_EDEVICE: return "HARP_EDEVICE: device-side check failed";
    }
    return "unknown harp_status";
}

int harp_last_cuda_error(void) { return (int)t_last_err; }

const char* harp_last_cuda_error_str(void) { return cudaGetErrorString(t_last_err); }

}  // extern "C"
