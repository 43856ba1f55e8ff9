// Batched counting (many graphs, one launch sequence): the disjoint union of the member CSRs is
// counted by the same pipeline as a single graph, with every anchor's statistics routed to its own
// graph (an occurrence of a connected 4-vertex motif never spans two members).  The work queues are
// therefore global over (graph, anchor) items and ordered heavy-first by rank, so thousands of
// graphs of uneven size share one persistent launch per kernel.  The whole sequence - union build,
// orientation, anchors, reductions, per-graph closure, and the copy of the counts to pinned host
// memory - is captured once into a CUDA graph and replayed on every count.
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "harp_internal.cuh"

namespace harp {
namespace {

struct MemberDesc {
    const int64_t* off;
    const int32_t* cols;
    int64_t n;
    int64_t vbase;   // first union vertex of this member
    int64_t abase;   // first union arc of this member
    int64_t bstart;  // first union-build block of this member
};

// Union-build blocks per member: one per kUnionChunk vertices or arcs, whichever needs more.
constexpr int64_t kUnionChunk = 16384;

int64_t union_blocks(int64_t n, int64_t arcs) {
    const int64_t x = n > arcs ? n : arcs;
    const int64_t b = (x + kUnionChunk - 1) / kUnionChunk;
    return b < 1 ? 1 : b;
}

// Block b copies chunk (b - bstart) of its member (found by binary search over bstart): shifted
// offsets and graph ids for that chunk of vertices, shifted columns for that chunk of arcs.
__global__ void __launch_bounds__(256) k_union_build(const MemberDesc* __restrict__ desc, int64_t G,
                                                     int64_t* __restrict__ off_u, int32_t* __restrict__ cols_u,
                                                     int32_t* __restrict__ gid_u, int64_t N, int64_t A) {
    int64_t lo = 0, hi = G;  // member: last g with desc[g].bstart <= blockIdx.x
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (desc[mid].bstart <= (int64_t)blockIdx.x) lo = mid;
        else hi = mid;
    }
    const int64_t g = lo;
    const MemberDesc d = desc[g];
    const int64_t c0 = ((int64_t)blockIdx.x - d.bstart) * kUnionChunk;
    const int64_t vend = c0 + kUnionChunk < d.n ? c0 + kUnionChunk : d.n;
    for (int64_t v = c0 + threadIdx.x; v < vend; v += blockDim.x) {
        off_u[d.vbase + v] = d.abase + d.off[v];
        gid_u[d.vbase + v] = (int32_t)g;
    }
    const int64_t arcs = d.n > 0 ? d.off[d.n] : 0;
    const int64_t aend = c0 + kUnionChunk < arcs ? c0 + kUnionChunk : arcs;
    for (int64_t a = c0 + threadIdx.x; a < aend; a += blockDim.x) cols_u[d.abase + a] = (int32_t)(d.vbase + d.cols[a]);
    if (blockIdx.x == 0 && threadIdx.x == 0) off_u[N] = A;
}

// Pinned host buffers for the batch outputs, kept for reuse: allocating and freeing page-locked
// memory synchronises the whole device, which would stall unrelated streams (a server building the
// next requests while a batch counts).
std::mutex g_pinned_mu;
std::multimap<size_t, void*> g_pinned_free;

cudaError_t pinned_get(size_t bytes, void** out) {
    {
        std::lock_guard<std::mutex> lk(g_pinned_mu);
        auto it = g_pinned_free.lower_bound(bytes);
        if (it != g_pinned_free.end() && it->first <= 4 * bytes + 4096) {
            *out = it->second;
            g_pinned_free.erase(it);
            return cudaSuccess;
        }
    }
    return cudaMallocHost(out, bytes);
}

void pinned_put(size_t bytes, void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (g_pinned_free.size() >= 64) {  // bound the cache: drop the smallest entry
        auto it = g_pinned_free.begin();
        cudaFreeHost(it->second);
        g_pinned_free.erase(it);
    }
    g_pinned_free.emplace(bytes, p);
}

}  // namespace
}  // namespace harp

using namespace harp;

struct harp_batch {
    int device = 0;
    cudaStream_t capture_stream = nullptr;
    int64_t G = 0;
    std::vector<int64_t> m_of;        // per-member m (host)
    harp_csr u;                       // the union (owns off/cols + workspace)
    MemberDesc* d_desc = nullptr;
    int32_t* d_gid_in = nullptr;      // [N]
    int32_t* d_gid = nullptr;         // [N]
    uint64_t* d_accG = nullptr;       // [G * kGStride]
    int64_t* d_gbase = nullptr;       // [G + 1] first union vertex of each member
    int64_t* d_ginfo = nullptr;       // [G * kGInfo]
    uint64_t* d_out = nullptr;        // [G * 16]
    uint64_t* h_out = nullptr;        // pinned [G * 16 + 1]; the last word is the device self-check flag
    size_t h_out_bytes = 0;           // capacity of h_out (from the pinned-buffer cache)
    cudaGraphExec_t exec = nullptr;
    harp_plan plan_captured{};
    int64_t launches_per_count = 0;
};

namespace {

harp_status batch_release(harp_batch* b) {
    if (!b) return HARP_OK;
    cudaSetDevice(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaStream_t s = b->capture_stream;
    ws_release(b->u.ws, s);
    if (b->u.off) cudaFreeAsync(b->u.off, s);
    if (b->u.cols) cudaFreeAsync(b->u.cols, s);
    if (b->d_desc) cudaFreeAsync(b->d_desc, s);
    if (b->d_gid_in) cudaFreeAsync(b->d_gid_in, s);
    if (b->d_gid) cudaFreeAsync(b->d_gid, s);
    if (b->d_accG) cudaFreeAsync(b->d_accG, s);
    if (b->d_gbase) cudaFreeAsync(b->d_gbase, s);
    if (b->d_ginfo) cudaFreeAsync(b->d_ginfo, s);
    if (b->d_out) cudaFreeAsync(b->d_out, s);
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (b->h_out) pinned_put(b->h_out_bytes, b->h_out);
    delete b;
    return HARP_OK;
}

// Enqueue the whole batched count on stream s (also used while capturing).
harp_status enqueue_batch(harp_batch* b, const harp_plan& plan, cudaStream_t s) {
    Workspace& ws = b->u.ws;
    HARP_CK(cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s));
    HARP_CK(cudaMemsetAsync(b->d_accG, 0, sizeof(uint64_t) * kGStride * (size_t)b->G, s));
    HARP_TRY(orient(&b->u, ws, s));
    HARP_TRY(count_triangles_k4(&b->u, ws, plan, s));
    HARP_TRY(count_wedge_c4(&b->u, ws, plan, s));
    HARP_TRY(reduce_and_close_batch(&b->u, ws, b->G, b->d_out, s));
    HARP_CK(cudaMemcpyAsync(b->h_out, b->d_out, sizeof(uint64_t) * 16 * (size_t)b->G, cudaMemcpyDeviceToHost, s));
    HARP_CK(cudaMemcpyAsync(b->h_out + 16 * b->G, ws.acc + ACC_ERR, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    return HARP_OK;
}

bool same_plan(const harp_plan& a, const harp_plan& b) {
    return a.basis == b.basis && a.tri_probe == b.tri_probe && a.tri_warp_max == b.tri_warp_max &&
           a.tri_cta_max == b.tri_cta_max && a.tri_big_max == b.tri_big_max &&
           a.c4_warp_max_work == b.c4_warp_max_work && a.c4_cta_max_work == b.c4_cta_max_work &&
           a.c4_window_bytes == b.c4_window_bytes && a.flags == b.flags &&
           a.tri_probe_bin[0] == b.tri_probe_bin[0] && a.tri_probe_bin[1] == b.tri_probe_bin[1] &&
           a.tri_probe_bin[2] == b.tri_probe_bin[2] && a.tri_probe_bin[3] == b.tri_probe_bin[3];
}

}  // namespace

extern "C" {

harp_status harp_batch_create(const harp_csr* const* graphs, int64_t G, harp_batch** out) {
    if (!out || G < 0 || (G > 0 && !graphs)) return HARP_EINVAL;
    int dev = 0;
    HARP_CK(cudaGetDevice(&dev));
    int64_t N = 0, M = 0, maxdeg = 0;
    for (int64_t g = 0; g < G; ++g) {
        if (!graphs[g]) return HARP_EINVAL;
        if (graphs[g]->device != dev) return HARP_EINVAL;
        N += graphs[g]->n;
        M += graphs[g]->m;
        if (graphs[g]->max_deg > maxdeg) maxdeg = graphs[g]->max_deg;
    }
    if (N > 2147483647LL || 2 * M > 4294967295LL || G > 2147483647LL) return HARP_EOVERFLOW;
    harp_batch* b = new (std::nothrow) harp_batch();
    if (!b) return HARP_ENOMEM;
    b->device = dev;
    b->G = G;
    b->m_of.resize((size_t)G);
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    cudaStream_t s = b->capture_stream;
    std::vector<MemberDesc> desc((size_t)G);
    std::vector<int64_t> gbase((size_t)G + 1);
    int64_t vb = 0, ab = 0, blocks = 0;
    for (int64_t g = 0; g < G; ++g) {
        const harp_csr* c = graphs[g];
        desc[(size_t)g] = MemberDesc{c->off, c->cols, c->n, vb, ab, blocks};
        gbase[(size_t)g] = vb;
        b->m_of[(size_t)g] = c->m;
        vb += c->n;
        ab += 2 * c->m;
        blocks += union_blocks(c->n, 2 * c->m);
    }
    gbase[(size_t)G] = vb;
    const size_t gg = (size_t)(G > 0 ? G : 1);
    b->u.device = dev;
    b->u.stream = s;
    b->u.n = N;
    b->u.m = M;
    b->u.max_deg = maxdeg;
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->u.off, sizeof(int64_t) * (size_t)(N + 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->u.cols, sizeof(int32_t) * (size_t)(2 * M > 0 ? 2 * M : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_desc, sizeof(MemberDesc) * gg, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_gid_in, sizeof(int32_t) * (size_t)(N > 0 ? N : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_gid, sizeof(int32_t) * (size_t)(N > 0 ? N : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_accG, sizeof(uint64_t) * kGStride * gg, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_out, sizeof(uint64_t) * 16 * gg, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_gbase, sizeof(int64_t) * (gg + 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_ginfo, sizeof(int64_t) * kGInfo * gg, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_gbase, gbase.data(), sizeof(int64_t) * (size_t)(G + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        b->h_out_bytes = sizeof(uint64_t) * (16 * gg + 1);
        e = pinned_get(b->h_out_bytes, (void**)&b->h_out);
    }
    if (e == cudaSuccess && G > 0)
        e = cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(MemberDesc) * (size_t)G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && blocks > 2147483647LL) e = cudaErrorInvalidValue;
    if (e == cudaSuccess && G == 0) e = cudaMemsetAsync(b->u.off, 0, sizeof(int64_t), s);  // off[0] = 0
    if (e == cudaSuccess && G > 0) {
        k_union_build<<<(unsigned)blocks, 256, 0, s>>>(b->d_desc, G, b->u.off, b->u.cols, b->d_gid_in, N, 2 * M);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // desc is a host vector: wait before it goes
    if (e != cudaSuccess) {
        record_cuda_error(e);
        batch_release(b);
        return e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
    }
    b->u.csr_bytes = sizeof(int64_t) * (size_t)(N + 1) + sizeof(int32_t) * (size_t)(2 * M);
    *out = b;
    return HARP_OK;
}

}  // extern "C"

namespace {

// Prepare b for counting under `plan`: workspace, batch pointers, and (unless the plan asks for
// direct launches) the CUDA graph of the whole sequence, captured again only when the plan changes.
harp_status batch_prepare(harp_batch* b, const harp_plan& plan) {
    HARP_TRY(ws_ensure(b->u.ws, b->u.n, b->u.m, b->capture_stream));
    b->u.ws.gid_in = b->d_gid_in;
    b->u.ws.gid = b->d_gid;
    b->u.ws.accG = b->d_accG;
    b->u.ws.G = b->G;
    b->u.ws.gbase = b->d_gbase;
    b->u.ws.ginfo = b->d_ginfo;
    const bool use_graph = !(plan.flags & HARP_PLAN_NO_GRAPH);
    if (use_graph && (!b->exec || !same_plan(plan, b->plan_captured))) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        HARP_CK(cudaStreamSynchronize(b->capture_stream));
        cudaGraph_t graph = nullptr;
        const int64_t l0 = harp_launch_count();
        HARP_CK(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed));
        harp_status st = enqueue_batch(b, plan, b->capture_stream);
        cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
        if (st != HARP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) {
            record_cuda_error(e);
            return HARP_ECUDA;
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            b->exec = nullptr;
            return HARP_ECUDA;
        }
        b->launches_per_count = harp_launch_count() - l0;
        b->plan_captured = plan;
    }
    return HARP_OK;
}

}  // namespace

extern "C" {

harp_status harp_batch_count(harp_batch* b, const harp_plan* user_plan, uint64_t (*counts_out)[6],
                             uint64_t (*stats_out)[8], void* stream) {
    if (!b || (!counts_out && b->G > 0)) return HARP_EINVAL;
    if (user_plan && user_plan->basis != HARP_BASIS_TRIANGLE_WEDGE) return HARP_EINVAL;
    HARP_CK(cudaSetDevice(b->device));
    cudaStream_t s = (cudaStream_t)stream;
    harp_plan plan;
    normalise_plan(user_plan, &plan);
    HARP_TRY(batch_prepare(b, plan));
    const bool use_graph = !(plan.flags & HARP_PLAN_NO_GRAPH);
    if (use_graph) {
        HARP_CK(cudaGraphLaunch(b->exec, s));
        note_launch(b->launches_per_count);
        HARP_CK(cudaStreamSynchronize(s));
    } else {
        HARP_CK(cudaStreamSynchronize(b->capture_stream));
        HARP_TRY(enqueue_batch(b, plan, s));
        HARP_CK(cudaStreamSynchronize(s));
    }
    if (b->h_out[16 * b->G]) return HARP_EDEVICE;  // a kernel's self-check skipped an out-of-range access
    for (int64_t g = 0; g < b->G; ++g) {
        const uint64_t* o = b->h_out + 16 * g;
        for (int k = 0; k < 6; ++k) counts_out[g][k] = o[k];
        if (stats_out) {
            for (int k = 0; k < 8; ++k) stats_out[g][k] = o[8 + k];
            stats_out[g][HARP_STAT_EDGES] = (uint64_t)b->m_of[(size_t)g];
        }
    }
    return HARP_OK;
}

void harp_batch_free(harp_batch* b) { batch_release(b); }

harp_status harp_batch_autotune(harp_batch* b, const harp_plan* candidates, int32_t ncand, int32_t reps,
                                harp_plan* best, float* ms_out) {
    if (!b || !best || reps < 1) return HARP_EINVAL;
    if (candidates && ncand < 1) return HARP_EINVAL;
    HARP_CK(cudaSetDevice(b->device));
    cudaStream_t s = b->capture_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HARP_CK(cudaEventCreate(&e0));
    HARP_CK(cudaEventCreate(&e1));
    std::vector<uint64_t> first;
    std::vector<harp_plan> timed;  // every plan timed so far and its time: identical plans run once
    std::vector<float> timed_ms;
    // time plan p (captured graph: one untimed replay, then reps timed); its counts must equal the
    // first candidate's
    auto time_plan = [&](const harp_plan& p, float* ms_res) -> harp_status {
        for (size_t k = 0; k < timed.size(); ++k)
            if (same_plan(timed[k], p)) {
                *ms_res = timed_ms[k];
                return HARP_OK;
            }
        HARP_TRY(batch_prepare(b, p));
        cudaError_t e = cudaGraphLaunch(b->exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int32_t r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            return HARP_ECUDA;
        }
        note_launch(b->launches_per_count * (reps + 1));
        if (b->h_out[16 * b->G]) return HARP_EDEVICE;
        // every candidate must produce the same counts and statistics (a plan changes only the work)
        std::vector<uint64_t> now(b->h_out, b->h_out + 16 * b->G);
        if (first.empty()) first = now;
        else if (now != first) return HARP_EDEVICE;
        ms /= (float)reps;
        if (ms_out && timed.size() < (size_t)(candidates ? ncand : HARP_AUTOTUNE_GRID)) ms_out[timed.size()] = ms;
        timed.push_back(p);
        timed_ms.push_back(ms);
        *ms_res = ms;
        return HARP_OK;
    };
    harp_status st = HARP_OK;
    harp_plan cur;
    if (candidates) {
        float best_ms = 0.0f;
        for (int32_t k = 0; k < ncand && st == HARP_OK; ++k) {
            if (candidates[k].basis != HARP_BASIS_TRIANGLE_WEDGE) {
                st = HARP_EINVAL;
                break;
            }
            harp_plan p;
            normalise_plan(&candidates[k], &p);
            p.flags &= ~HARP_PLAN_NO_GRAPH;  // candidates are timed as captured graphs
            float ms = 0.0f;
            st = time_plan(p, &ms);
            if (st == HARP_OK && (k == 0 || ms < best_ms)) {
                best_ms = ms;
                cur = p;
            }
        }
    } else {
        // per-degree-bin coordinate descent from the default plan: each knob in turn takes the value
        // that times fastest with the others held at their current best
        if (ms_out)
            for (int k = 0; k < HARP_AUTOTUNE_GRID; ++k) ms_out[k] = 0.0f;
        normalise_plan(nullptr, &cur);
        float cur_ms = 0.0f;
        st = time_plan(cur, &cur_ms);
        auto try_knob = [&](auto set, std::initializer_list<uint32_t> values) {
            for (uint32_t v : values) {
                if (st != HARP_OK) return;
                harp_plan p = cur;
                set(p, v);
                float ms = 0.0f;
                st = time_plan(p, &ms);
                if (st == HARP_OK && ms < cur_ms) {
                    cur = p;
                    cur_ms = ms;
                }
            }
        };
        try_knob([](harp_plan& p, uint32_t v) { p.tri_warp_max = v; }, {16u, 32u});
        for (int bin = 0; bin < 4; ++bin)
            try_knob([bin](harp_plan& p, uint32_t v) { p.tri_probe_bin[bin] = (uint8_t)v; },
                     {(uint32_t)HARP_PROBE_HASH, (uint32_t)HARP_PROBE_BSEARCH});
        try_knob([](harp_plan& p, uint32_t v) { p.tri_cta_max = v; }, {256u, 512u, 1024u});
        try_knob([](harp_plan& p, uint32_t v) { p.c4_warp_max_work = v; }, {256u, 512u});
        try_knob([](harp_plan& p, uint32_t v) { p.c4_window_bytes = v; }, {100u * 1024u, 200u * 1024u});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HARP_OK) return st;
    *best = cur;
    return HARP_OK;
}

harp_status harp_batch_info(const harp_batch* b, int64_t* graphs, int64_t* n_total, int64_t* m_total,
                            size_t* device_bytes) {
    if (!b) return HARP_EINVAL;
    if (graphs) *graphs = b->G;
    if (n_total) *n_total = b->u.n;
    if (m_total) *m_total = b->u.m;
    if (device_bytes)
        *device_bytes = b->u.csr_bytes + b->u.ws.bytes + (size_t)b->u.n * 8 + (size_t)b->G * (kGStride + 16) * 8;
    return HARP_OK;
}

harp_status harp_count4_batch(const harp_csr* const* graphs, int64_t G, const harp_plan* plan,
                              uint64_t (*counts_out)[6], void* stream) {
    harp_batch* b = nullptr;
    HARP_TRY(harp_batch_create(graphs, G, &b));
    harp_plan p;
    normalise_plan(plan, &p);
    p.flags |= HARP_PLAN_NO_GRAPH;  // one count: capturing a graph would not pay for itself
    const harp_status st = harp_batch_count(b, &p, counts_out, nullptr, stream);
    batch_release(b);
    return st;
}

}  // extern "C"
