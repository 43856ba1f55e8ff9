// Step a2: anchor selection (Section III-A, Eq. 1) and closure-driven synthesis (Section III-B).
//
//   B* = argmin_B [ C_enum(B) + l_I C_inter(B) + l_H C_halo(B) - l_R R_reuse(B) - l_Y Y_closure(B) ]
//
// The two legal anchor families for connected 4-vertex motifs are scored from a uniform sample of
// arcs (u, v) of the graph, for each of which one warp computes d_u, d_v and the exact common
// neighbour count t_uv (the intersection of the two sorted rows):
//   * TW  (triangle + per-edge t_e + 4-clique extension + ordered wedges, Section III-B):
//         C_enum = wedge work ~ sum_e min(d_u, d_v); C_inter = oriented 2-path probes ~ the same;
//         R_reuse = 4-clique extensions answered by a staged frontier (one per triangle, each saving
//         a walk of ~min(d_u, d_v)).
//   * LIT (the closure equations as printed, Section III-F: per-triangle X_j, per-edge A_e x B_e,
//         per-vertex H_u): C_enum = the row intersections of every arc plus, per triangle, the
//         three-way intersection for X_3, and per edge one frontier per x in A_e; C_inter = the
//         signature-cache probes; R_reuse = frontier requests expected to hit the cache.
// Both also pay a fixed cost per kernel launch after the shared orientation pass (15 for TW, 4 for
// LIT), expressed in element operations: kLaunchOps, about the element operations one dependent
// launch costs at the measured rate of the wedge kernel (~4e11 elements/s, ~2.5 us a launch).  Both
// recover all six counts (Y = 6).  The lambda weights normalise the terms to element operations (the
// paper leaves their values open): l_I = 1, l_H = 1/4 per replicated byte, l_R = 1 (reuse is counted
// in the element operations it saves), l_Y = 0 (equal yield decides nothing between these bases).
// The plan never changes the counts.
//
// The same sample chooses the execution-mode thresholds (warp-local vs CTA, Section III-D).
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>

#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kSampleThreads = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// One warp per sample i: a uniform arc a in [0, 2m), its endpoints u (row) and v, their degrees and
// t_uv = |N(u) n N(v)| (lanes walk the shorter row and binary-search the longer).
// out[3 * i + 0] = d_u, [+1] = d_v, [+2] = t_uv.
__global__ void k_plan_sample(const int64_t* __restrict__ off, const int32_t* __restrict__ cols, int64_t n,
                              int64_t arcs, uint64_t samples, uint64_t seed, uint32_t* __restrict__ out) {
    const int l = lane_id();
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < samples; i += nw) {
        const uint64_t a = mix64(seed + 0x9E3779B97F4A7C15ULL * (i + 1)) % (uint64_t)arcs;
        int64_t lo = 0, hi = n;  // last row with off[row] <= a
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if ((uint64_t)off[mid] <= a) lo = mid;
            else hi = mid;
        }
        const int64_t u = lo;
        const int32_t v = cols[a];
        const int64_t ub = off[u], ue = off[u + 1], vb = off[v], ve = off[v + 1];
        const bool ushort = ue - ub <= ve - vb;
        const int64_t sb = ushort ? ub : vb, se = ushort ? ue : ve;
        const int64_t lb = ushort ? vb : ub, le = ushort ? ve : ue;
        uint32_t t = 0;
        for (int64_t k = sb + l; k < se; k += 32) {
            const int32_t x = cols[k];
            const int64_t p = lb + lower_bound_i32(cols + lb, le - lb, x);
            t += (p < le && cols[p] == x) ? 1u : 0u;
        }
        t = warp_sum(t);
        if (l == 0) {
            out[3 * i] = (uint32_t)(ue - ub);
            out[3 * i + 1] = (uint32_t)(ve - vb);
            out[3 * i + 2] = t;
        }
    }
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
    p->c4_cta_max_work = 2048;
    p->c4_window_bytes = 0;  // by graph size (count_wedge_c4)
    p->flags = 0;
    p->est_halo = 1.0;
    p->est_yield = 6.0;
    p->lit_cache_log2 = 0;
    p->lit_cache_min_deg = 0;
    for (int k = 0; k < 4; ++k) p->tri_probe_bin[k] = (uint8_t)HARP_PROBE_HASH;
}

size_t plan_bytes(const harp_plan* p) {
    if (p && p->version == 1) return offsetof(harp_plan, lit_cache_log2);
    return sizeof(harp_plan);
}

void normalise_plan(const harp_plan* user, harp_plan* out) {
    default_plan(out);
    if (!user) return;
    harp_plan in;  // a version-1 plan stops before the cache fields: they keep their defaults
    default_plan(&in);
    std::memcpy(&in, user, plan_bytes(user));
    out->basis = in.basis;
    if (in.tri_probe) out->tri_probe = in.tri_probe;
    if (in.tri_warp_max) out->tri_warp_max = in.tri_warp_max > 32 ? 32 : in.tri_warp_max;
    if (in.tri_cta_max) out->tri_cta_max = in.tri_cta_max > 1024 ? 1024 : in.tri_cta_max;
    if (in.tri_big_max) out->tri_big_max = in.tri_big_max > 4096 ? 4096 : in.tri_big_max;
    if (in.c4_warp_max_work) out->c4_warp_max_work = in.c4_warp_max_work;
    if (in.c4_cta_max_work) out->c4_cta_max_work = in.c4_cta_max_work;
    if (in.c4_window_bytes) out->c4_window_bytes = in.c4_window_bytes;
    out->flags = in.flags;
    out->est_enum = in.est_enum;
    out->est_inter = in.est_inter;
    out->est_halo = in.est_halo;
    out->est_reuse = in.est_reuse;
    out->est_yield = in.est_yield;
    out->objective = in.objective;
    out->lit_cache_log2 = in.lit_cache_log2 > 30 ? 30 : in.lit_cache_log2;
    out->lit_cache_min_deg = in.lit_cache_min_deg;
    for (int k = 0; k < 4; ++k)  // a bin's probe, else the plan-wide one
        out->tri_probe_bin[k] = (in.tri_probe_bin[k] == HARP_PROBE_HASH || in.tri_probe_bin[k] == HARP_PROBE_BSEARCH)
                                    ? in.tri_probe_bin[k]
                                    : (uint8_t)out->tri_probe;
    out->est_cost_tw = in.est_cost_tw;
    out->est_cost_lit = in.est_cost_lit;
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
    // per-sample (d_u, d_v, t_uv) of uniform arcs, exact
    uint32_t* host = nullptr;
    uint64_t got = 0;
    if (g->m > 0) {
        HARP_CK(cudaSetDevice(g->device));
        host = new (std::nothrow) uint32_t[3 * samples];
        if (!host) return HARP_ENOMEM;
        uint32_t* d_smp = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&d_smp, 3 * samples * sizeof(uint32_t), g->stream);
        if (e == cudaSuccess) {
            const uint64_t blocks = (samples * 32 + 255) / 256;
            k_plan_sample<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, g->stream>>>(
                g->off, g->cols, g->n, 2 * g->m, samples, seed, d_smp);
            note_launch();
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(host, d_smp, 3 * samples * sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream);
            cudaFreeAsync(d_smp, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        }
        if (e != cudaSuccess) {
            delete[] host;
            record_cuda_error(e);
            return HARP_ECUDA;
        }
        got = samples;
    }
    const double mean_deg = g->n > 0 ? 2.0 * m / (double)g->n : 0.0;
    // per-arc means of the cost terms (element operations); lg = binary-search depth in the longer row
    double tw_enum = 0, tw_inter = 0, tw_reuse = 0, lit_enum = 0, lit_inter = 0, lit_reuse = 0;
    for (uint64_t i = 0; i < got; ++i) {
        const double du = host[3 * i], dv = host[3 * i + 1], t = host[3 * i + 2];
        const double dl = du < dv ? du : dv, dh = du < dv ? dv : du;
        const double lg = std::log2(dh + 2.0);
        const double A = dl - 1.0 - t > 0 ? dl - 1.0 - t : 0.0;  // |A_e| from the lower-degree end
        tw_enum += dl;                  // ordered wedges through the edge, about min(d_u, d_v)
        tw_inter += dl;                 // oriented 2-path probes
        tw_reuse += (t / 3.0) * dl;     // one staged 4-clique extension per triangle (t/3 per edge)
        // literal: the arc's intersection (tri pass and edge pass), the X_3 walks of its t/3
        // triangles, and per x in A_e the correction |C_e n N(x)| plus a frontier (half of them
        // computed on a miss, at min(d_x, d_v) with d_x ~ the mean degree)
        lit_enum += 2.0 * dl * lg + (t / 3.0) * t * lg + A * (t * lg + 0.5 * std::fmin(mean_deg, dh) * lg);
        lit_inter += 2.0 * (t / 3.0) + A + 2.0;  // cache probes: two per triangle, one per x, two per edge
        lit_reuse += 0.5 * A * std::fmin(mean_deg, dh) * lg;  // frontier hits save their recompute
    }
    delete[] host;
    const double inv = got > 0 ? 1.0 / (double)got : 0.0;
    tw_enum *= m * inv;
    tw_inter *= m * inv;
    tw_reuse *= m * inv;
    lit_enum *= m * inv;
    lit_inter *= m * inv;
    lit_reuse *= m * inv;
    // fixed cost of the kernel launches after the shared orientation pass
    constexpr double kLaunchOps = 1.0e6;
    tw_enum += 15.0 * kLaunchOps;
    lit_enum += 4.0 * kLaunchOps;
    // Halo term: replication factor if the CSR plus workspace exceed the memory budget.
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double budget = (opts && opts->memory_budget) ? (double)opts->memory_budget : (double)free_b;
    const double need = 8.0 * (double)(g->n + 1) * 3 + 4.0 * m * 6;
    const double halo = need > budget && budget > 0 ? 1.0 + need / budget : 1.0;
    const double lI = (opts && opts->lambda_inter > 0) ? opts->lambda_inter : 1.0;
    const double lH = (opts && opts->lambda_halo > 0) ? opts->lambda_halo : 0.25;
    const double lR = (opts && opts->lambda_reuse > 0) ? opts->lambda_reuse : 1.0;
    const double lY = (opts && opts->lambda_yield > 0) ? opts->lambda_yield : 0.0;
    const double J_tw = tw_enum + lI * tw_inter + lH * (halo - 1.0) * 4.0 * m - lR * tw_reuse - lY * 6.0;
    // the literal basis also keeps its signature cache (16 bytes a slot, 4m slots) on the device
    const double J_lit = lit_enum + lI * lit_inter + lH * (halo - 1.0) * 8.0 * m - lR * lit_reuse - lY * 6.0;
    const bool lit = got > 0 && J_lit < J_tw;
    p.basis = lit ? HARP_BASIS_LITERAL : HARP_BASIS_TRIANGLE_WEDGE;
    p.est_enum = lit ? lit_enum : tw_enum;
    p.est_inter = lit ? lit_inter : tw_inter;
    p.est_halo = halo;
    p.est_reuse = lit ? (lit_inter > 0 ? 0.5 * lit_inter / (lit_inter + m) : 0.0) : (tw_enum > 0 ? tw_reuse / tw_enum : 0.0);
    p.est_yield = 6.0;
    p.objective = lit ? J_lit : J_tw;
    p.est_cost_tw = J_tw;
    p.est_cost_lit = J_lit;
    // Execution-mode thresholds: light graphs keep more roots in warp-local mode.
    p.c4_warp_max_work = mean_deg < 8 ? 512 : 256;
    p.c4_cta_max_work = 2048;
    // out->version picks the layout written: 1 = a version-1 plan (ends at `objective`), else current
    if (out->version == 1) p.version = 1;
    std::memcpy(out, &p, plan_bytes(&p));
    return HARP_OK;
}
