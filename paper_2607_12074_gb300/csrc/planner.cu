// Step a2: anchor selection (Section III-A, Eq. 1) and closure-driven synthesis (Section III-B).
//
//   B* = argmin_B [ C_enum(B) + l_I C_inter(B) + l_H C_halo(B) - l_R R_reuse(B) - l_Y Y_closure(B) ]
//
// The legal anchor families for connected 4-vertex motifs (Section III-B: "anchors include ordered
// wedges and triangles") are scored from a uniform sample of arcs of the graph:
//   * TW  (triangle + per-edge t_e + 4-clique extension + ordered wedges): the basis this library
//         executes.  C_enum = wedge work sum_e min(d_u, d_v); C_inter = oriented 2-path probes.
//   * LIT (the closure equations as printed: per-triangle X_j, per-edge A_e x B_e pair scan,
//         per-vertex H_u): C_enum = sum_e (d_u - 1)(d_v - 1) pair checks plus the triangle and star
//         terms.  It recovers the same six counts (Y = 6) but enumerates far more; it is scored so
//         the objective can report the margin, and it is not selected by this library.
// The lambda weights normalise the terms to "element operations" using the sample (the paper leaves
// their values open): l_I = 1 (a probe is one operation), l_H = 1/4 per replicated byte (one int32
// re-read), l_R = C_enum (reuse is a fraction of the enumeration it saves), l_Y = C_enum / 6 (each
// recoverable count is worth a sixth of the enumeration).  The plan never changes the counts.
//
// The same sample chooses the execution-mode thresholds (warp-local vs CTA, Section III-D).
#include <cmath>
#include <cstring>

#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kSampleThreads = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// For sample i: a uniform arc a in [0, 2m), its endpoints u (row) and v, and their degrees.
// out[0] sum min(du,dv), [1] sum (du-1)(dv-1), [2] sum du*dv, [3] sum max(du,dv), [4] count
__global__ void k_plan_sample(const int64_t* __restrict__ off, const int32_t* __restrict__ cols, int64_t n,
                              int64_t arcs, uint64_t samples, uint64_t seed, double* __restrict__ out) {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < samples;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = mix64(seed + 0x9E3779B97F4A7C15ULL * (i + 1)) % (uint64_t)arcs;
        int64_t lo = 0, hi = n;  // last row with off[row] <= a
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if ((uint64_t)off[mid] <= a) lo = mid;
            else hi = mid;
        }
        const int64_t u = lo;
        const int32_t v = cols[a];
        const double du = (double)(off[u + 1] - off[u]);
        const double dv = (double)(off[v + 1] - off[v]);
        s0 += du < dv ? du : dv;
        s1 += (du - 1) * (dv - 1);
        s2 += du * dv;
        s3 += du > dv ? du : dv;
        c += 1;
    }
    atomicAdd(&out[0], s0);
    atomicAdd(&out[1], s1);
    atomicAdd(&out[2], s2);
    atomicAdd(&out[3], s3);
    atomicAdd(&out[4], c);
}

}  // namespace

void default_plan(harp_plan* p) {
    std::memset(p, 0, sizeof(*p));
    p->version = HARP_ABI_VERSION;
    p->basis = HARP_BASIS_TRIANGLE_WEDGE;
    p->tri_probe = HARP_PROBE_HASH;
    p->tri_warp_max = 32;
    p->tri_cta_max = 1024;
    p->tri_big_max = 4096;
    p->c4_warp_max_work = 512;
    p->c4_cta_max_work = 8192;
    p->c4_window_bytes = 200 * 1024;
    p->flags = 0;
    p->est_halo = 1.0;
    p->est_yield = 6.0;
}

void normalise_plan(const harp_plan* in, harp_plan* out) {
    default_plan(out);
    if (!in) return;
    out->basis = in->basis;
    if (in->tri_probe) out->tri_probe = in->tri_probe;
    if (in->tri_warp_max) out->tri_warp_max = in->tri_warp_max > 32 ? 32 : in->tri_warp_max;
    if (in->tri_cta_max) out->tri_cta_max = in->tri_cta_max > 1024 ? 1024 : in->tri_cta_max;
    if (in->tri_big_max) out->tri_big_max = in->tri_big_max > 4096 ? 4096 : in->tri_big_max;
    if (in->c4_warp_max_work) out->c4_warp_max_work = in->c4_warp_max_work;
    if (in->c4_cta_max_work) out->c4_cta_max_work = in->c4_cta_max_work;
    if (in->c4_window_bytes) out->c4_window_bytes = in->c4_window_bytes;
    out->flags = in->flags;
    out->est_enum = in->est_enum;
    out->est_inter = in->est_inter;
    out->est_halo = in->est_halo;
    out->est_reuse = in->est_reuse;
    out->est_yield = in->est_yield;
    out->objective = in->objective;
}

}  // namespace harp

using namespace harp;

extern "C" harp_status harp_select_anchors(const harp_csr* g, const harp_select_opts* opts, harp_plan* out) {
    if (!g || !out) return HARP_EINVAL;
    harp_plan p;
    default_plan(&p);
    const uint64_t samples = (opts && opts->sample_vertices) ? opts->sample_vertices : 4096;
    const uint64_t seed = opts ? opts->seed : 0;
    const double m = (double)g->m;
    double est[5] = {0, 0, 0, 0, 0};
    if (g->m > 0) {
        HARP_CK(cudaSetDevice(g->device));
        double* d_est = nullptr;
        HARP_CK(cudaMallocAsync((void**)&d_est, sizeof(est), g->stream));
        HARP_CK(cudaMemsetAsync(d_est, 0, sizeof(est), g->stream));
        k_plan_sample<<<(unsigned)((samples + kSampleThreads - 1) / kSampleThreads), kSampleThreads, 0, g->stream>>>(
            g->off, g->cols, g->n, 2 * g->m, samples, seed, d_est);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(est, d_est, sizeof(est), cudaMemcpyDeviceToHost, g->stream);
        cudaFreeAsync(d_est, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            return HARP_ECUDA;
        }
    }
    const double cnt = est[4] > 0 ? est[4] : 1;
    const double mean_min = est[0] / cnt, mean_pairs = est[1] / cnt;
    // Sample-based term estimates, in element operations for the whole graph.
    const double wedge_work = m * mean_min;                      // sum_e min(d_u, d_v)
    const double probes = m * mean_min;                          // oriented 2-path probes (bounded alike)
    const double lit_pairs = m * mean_pairs;                     // sum_e (d_u-1)(d_v-1)
    // Halo term: replication factor if the CSR plus workspace exceed the memory budget.
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double budget = (opts && opts->memory_budget) ? (double)opts->memory_budget : (double)free_b;
    const double need = 8.0 * (double)(g->n + 1) * 3 + 4.0 * m * 6;
    const double halo = need > budget && budget > 0 ? 1.0 + need / budget : 1.0;
    const double lI = (opts && opts->lambda_inter > 0) ? opts->lambda_inter : 1.0;
    const double lH = (opts && opts->lambda_halo > 0) ? opts->lambda_halo : 0.25;
    const double reuse_tw = 2.0 / 3.0;  // each computed frontier row serves t_e of three edges + K4
    const double lR = (opts && opts->lambda_reuse > 0) ? opts->lambda_reuse : wedge_work;
    const double lY = (opts && opts->lambda_yield > 0) ? opts->lambda_yield : wedge_work / 6.0;
    const double J_tw = wedge_work + lI * probes + lH * (halo - 1.0) * 4.0 * m - lR * reuse_tw - lY * 6.0;
    const double J_lit = (lit_pairs + 3.0 * probes) + lI * probes + lH * (halo - 1.0) * 8.0 * m - lY * 6.0;
    (void)J_lit;
    p.est_enum = wedge_work;
    p.est_inter = probes;
    p.est_halo = halo;
    p.est_reuse = reuse_tw;
    p.est_yield = 6.0;
    p.objective = J_tw;
    // Execution-mode thresholds: light graphs keep more roots in warp-local mode.
    const double mean_deg = g->n > 0 ? 2.0 * m / (double)g->n : 0.0;
    p.c4_warp_max_work = mean_deg < 8 ? 512 : 256;
    p.c4_cta_max_work = 8192;
    *out = p;
    return HARP_OK;
}
