// Batched counting (many graphs, one launch sequence): the disjoint union of the member CSRs is
// counted by the same pipeline as a single graph, with every anchor's statistics routed to its own
// graph (an occurrence of a connected 4-vertex motif never spans two members).  The work queues are
// therefore global over (graph, anchor) items and ordered heavy-first by rank, so thousands of
// graphs of uneven size share one persistent launch per kernel.  The whole sequence - union build,
// orientation, anchors, reductions, per-graph closure, and the copy of the counts to pinned host
// memory - is captured once into a CUDA graph and replayed on every count.
#include <cstring>
#include <new>
#include <vector>

#include "harp_internal.cuh"

namespace harp {
namespace {

struct MemberDesc {
    const int64_t* off;
    const int32_t* cols;
    int64_t n;
    int64_t vbase;  // first union vertex of this member
    int64_t abase;  // first union arc of this member
};

// one block per member (grid-stride over members): shifted offsets, graph ids, shifted columns
__global__ void __launch_bounds__(256) k_union_build(const MemberDesc* __restrict__ desc, int64_t G,
                                                     int64_t* __restrict__ off_u, int32_t* __restrict__ cols_u,
                                                     int32_t* __restrict__ gid_u, int64_t N, int64_t A) {
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
        const MemberDesc d = desc[g];
        for (int64_t v = threadIdx.x; v < d.n; v += blockDim.x) {
            off_u[d.vbase + v] = d.abase + d.off[v];
            gid_u[d.vbase + v] = (int32_t)g;
        }
        const int64_t arcs = d.n > 0 ? d.off[d.n] : 0;
        for (int64_t a = threadIdx.x; a < arcs; a += blockDim.x)
            cols_u[d.abase + a] = (int32_t)(d.vbase + d.cols[a]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off_u[N] = A;
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
    if (b->h_out) cudaFreeHost(b->h_out);
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
           a.tri_cta_max == b.tri_cta_max &&
           a.c4_warp_max_work == b.c4_warp_max_work && a.c4_cta_max_work == b.c4_cta_max_work &&
           a.c4_window_bytes == b.c4_window_bytes && a.flags == b.flags;
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
    int64_t vb = 0, ab = 0;
    for (int64_t g = 0; g < G; ++g) {
        const harp_csr* c = graphs[g];
        desc[(size_t)g] = MemberDesc{c->off, c->cols, c->n, vb, ab};
        gbase[(size_t)g] = vb;
        b->m_of[(size_t)g] = c->m;
        vb += c->n;
        ab += 2 * c->m;
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
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_out, sizeof(uint64_t) * (16 * gg + 1));
    if (e == cudaSuccess && G > 0)
        e = cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(MemberDesc) * (size_t)G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        int64_t blocks = G < 152 * 16 ? G : 152 * 16;
        if (blocks < 1) blocks = 1;
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

harp_status harp_batch_count(harp_batch* b, const harp_plan* user_plan, uint64_t (*counts_out)[6],
                             uint64_t (*stats_out)[8], void* stream) {
    if (!b || (!counts_out && b->G > 0)) return HARP_EINVAL;
    if (user_plan && user_plan->basis != HARP_BASIS_TRIANGLE_WEDGE) return HARP_EINVAL;
    HARP_CK(cudaSetDevice(b->device));
    cudaStream_t s = (cudaStream_t)stream;
    harp_plan plan;
    normalise_plan(user_plan, &plan);
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
