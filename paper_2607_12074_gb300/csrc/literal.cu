// The literal anchor basis: the closure equations of Section III-F executed as printed, with the
// induced-signature cache of Section III-C (Eq. 2) for the frontiers they read.
//
//   triangles T = {a, b, c}:  X_j(T) = # vertices outside T adjacent to exactly j of a, b, c
//                             N_paw = sum X_1,  N_diamond = sum X_2 / 2,  N_clique4 = sum X_3 / 4
//   edges e = (u, v):         C_e = N(u) n N(v),  A_e = N(u) \ (C_e u {v}),  B_e = N(v) \ (C_e u {u})
//                             N_path4 = sum_e #{(x, y) in A_e x B_e : x !~ y}
//                             N_cycle4 = 1/4 sum_e #{(x, y) in A_e x B_e : x ~ y}
//   vertices u, H_u = G[N(u)]: N_star = sum_u C(d,3) - m(H_u)(d - 2) + sum_{v in N(u)} C(deg_H v, 2) - tau(H_u)
//
// Everything runs after the shared orientation pass (relabelled, row-sorted CSR in rank order:
// rows are sorted, degrees grow with rank).  Three passes, each one warp per anchor:
//   1. k_lit_tri, one warp per out-arc (u, v), u < v.  The frontier C_uv = N(u) n N(v) is computed
//      by walking N(u) (the shorter row: d_u <= d_v in rank order) against N(v), staged in shared
//      memory, and its size t_uv = |C_uv| = deg_H(v) in H_u is put in the signature cache.  Every
//      triangle (u, v, w) with w in C_uv above v is anchored here once; for it
//         X_3 = |C_uv n N(w)|                     (the staged frontier probed against N(w))
//         X_2 = (t_uv - 1) + (t_uw - 1) + (t_vw - 1) - 3 X_3
//         X_1 = (d_u + d_v + d_w - 6) - 2 X_2 - 3 X_3
//      with t_uw, t_vw read through the cache.  X_3(T) is also added to tau3[a] for a in T, since
//      tau(H_a) = (1/3) sum_{T containing a} X_3(T) (each 4-clique on a holds 3 of a's triangles).
//   2. k_lit_edge, one warp per out-arc (u, v): |A_e| = d_u - 1 - t_uv, |B_e| = d_v - 1 - t_uv and
//      the A_e x B_e pairs that are edges, E_e = sum_{x in A_e} |N(x) n B_e| with
//         |N(x) n B_e| = |N(x) n N(v)| - 1 - |C_uv n N(x)|
//      (u is a common neighbour of x and v; the rest of N(x) n N(v) n N[u] lies in C_uv).  The
//      frontier N(x) n N(v) of the non-adjacent pair (x, v) recurs for every common neighbour of x
//      and v that anchors an edge, so it is read through the cache; the correction probes the staged
//      C_uv.  path4 terms |A_e||B_e| - E_e, cycle4 terms E_e.
//   3. k_lit_star, one warp per vertex u: deg_H(v) = t_uv for every v in N(u) through the cache,
//      m(H_u) = (1/2) sum t_uv, tau(H_u) = tau3[u] / 3.
// The sums divided by 2 and 4 are accumulated in 128 bits, so the divisions are exact (a sum that is
// not divisible raises kErrLitDiv: it cannot happen for a simple graph).
//
// Signature cache (Section III-C).  A cached state is a 2-vertex partial embedding (j = 2) with
// generator ranks (a < b, 31 bits each) and a mask code saying which adjacency the completion
// requires and forbids: SIG_C = M+ {a, b}, M- {} on an edge a ~ b (the frontier C_ab of the triangle
// and edge closures); SIG_W = M+ {a, b}, M- {a ~ b} on a non-adjacent pair (the frontier of the
// 4-cycle closure through A_e x B_e).  The two codes share the raw candidate set definition
// N(a) n N(b) but never one entry: the mask keeps the states apart.  The key packs (code, a, b) into
// 64 bits; the value is the frontier's cardinality.  The table is open addressing over 2^k slots of
// (key, value) with a bounded probe window; insertion claims an empty slot with a CAS and publishes
// the value with a valid bit, so a reader that sees the key before its value treats it as a miss.
// Frontiers of pairs below the degree bin lit_cache_min_deg are recomputed instead of cached.  With
// the cache off (HARP_PLAN_NO_REUSE) every frontier is recomputed; the counts are the same.
#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kLitThreads = 256;
constexpr int kLitWarps = kLitThreads / 32;
constexpr int kStageCap = 512;        // C_uv members staged per warp (shared memory); larger: unstaged
constexpr int kProbeWindow = 16;      // cache slots probed per lookup / insertion
constexpr unsigned long long kSigEmpty = ~0ull;
constexpr unsigned long long kValid = 1ull << 32;
enum : uint64_t { SIG_C = 1, SIG_W = 2 };

struct SigCache {
    unsigned long long* keys;  // [mask + 1]
    unsigned long long* vals;  // [mask + 1]: kValid | value
    uint32_t mask;             // slots - 1; 0 = cache off
    int32_t min_deg;           // admission: both generator degrees >= min_deg
};

struct Graph {
    const int64_t* off;   // rank-order CSR, rows sorted
    const int32_t* cols;
    const int32_t* deg;
};

__device__ __forceinline__ uint64_t sig_key(uint64_t code, int32_t a, int32_t b) {
    const uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
    return (code << 62) | ((uint64_t)lo << 31) | (uint64_t)hi;
}

__device__ __forceinline__ uint32_t sig_slot(uint64_t k, uint32_t mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    return (uint32_t)k & mask;
}

__device__ __forceinline__ bool sig_find(const SigCache& c, uint64_t key, uint32_t& val) {
    uint32_t h = sig_slot(key, c.mask);
    for (int p = 0; p < kProbeWindow; ++p) {
        const unsigned long long k = *(volatile const unsigned long long*)&c.keys[h];
        if (k == key) {
            const unsigned long long v = *(volatile const unsigned long long*)&c.vals[h];
            if (!(v & kValid)) return false;  // claimed, value not yet published
            val = (uint32_t)v;
            return true;
        }
        if (k == kSigEmpty) return false;
        h = (h + 1) & c.mask;
    }
    return false;
}

__device__ __forceinline__ void sig_put(const SigCache& c, uint64_t key, uint32_t val) {
    uint32_t h = sig_slot(key, c.mask);
    for (int p = 0; p < kProbeWindow; ++p) {
        const unsigned long long prev = atomicCAS(&c.keys[h], kSigEmpty, (unsigned long long)key);
        if (prev == kSigEmpty || prev == key) {
            atomicExch(&c.vals[h], kValid | (unsigned long long)val);
            return;
        }
        h = (h + 1) & c.mask;
    }
    // the probe window is full: this frontier stays uncached
}

// first index in the sorted row [b, e) of cols with cols[i] >= x
__device__ __forceinline__ int64_t row_lb(const int32_t* __restrict__ cols, int64_t b, int64_t e, int32_t x) {
    return b + lower_bound_i32(cols + b, e - b, x);
}
__device__ __forceinline__ bool row_has(const int32_t* __restrict__ cols, int64_t b, int64_t e, int32_t x) {
    const int64_t p = row_lb(cols, b, e, x);
    return p < e && __ldg(cols + p) == x;
}

// |N(a) n N(b)| by one thread: walk the shorter row, binary-search the longer
__device__ uint32_t common_serial(const Graph& G, int32_t a, int32_t b) {
    int64_t ab = G.off[a], ae = G.off[a + 1], bb = G.off[b], be = G.off[b + 1];
    if (ae - ab > be - bb) {
        int64_t t = ab; ab = bb; bb = t;
        t = ae; ae = be; be = t;
    }
    uint32_t c = 0;
    for (int64_t k = ab; k < ae; ++k) c += row_has(G.cols, bb, be, __ldg(G.cols + k)) ? 1u : 0u;
    return c;
}

// |N(a) n N(b)| by the whole warp (result in every lane)
__device__ uint32_t common_warp(const Graph& G, int32_t a, int32_t b) {
    int64_t ab = G.off[a], ae = G.off[a + 1], bb = G.off[b], be = G.off[b + 1];
    if (ae - ab > be - bb) {
        int64_t t = ab; ab = bb; bb = t;
        t = ae; ae = be; be = t;
    }
    uint32_t c = 0;
    for (int64_t k = ab + lane_id(); k < ae; k += 32) c += row_has(G.cols, bb, be, __ldg(G.cols + k)) ? 1u : 0u;
    return warp_sum(c);
}

// Running counters of one thread: frontier requests and cache hits.
struct SigStats {
    uint64_t lookups = 0, hits = 0;
};

__device__ __forceinline__ bool cacheable(const SigCache& c, const Graph& G, int32_t a, int32_t b) {
    return c.mask != 0 && G.deg[a] >= c.min_deg && G.deg[b] >= c.min_deg;
}

// The frontier |N(a) n N(b)| of state `code`, by one thread: the cache, else computed (and cached).
__device__ uint32_t frontier_serial(const SigCache& c, const Graph& G, uint64_t code, int32_t a, int32_t b,
                                    SigStats& st) {
    ++st.lookups;
    const bool cached = cacheable(c, G, a, b);
    const uint64_t key = sig_key(code, a, b);
    uint32_t v = 0;
    if (cached && sig_find(c, key, v)) {
        ++st.hits;
        return v;
    }
    v = common_serial(G, a, b);
    if (cached) sig_put(c, key, v);
    return v;
}

// The same by the whole warp (lane 0 holds the statistics; every lane gets the value).
__device__ uint32_t frontier_warp(const SigCache& c, const Graph& G, uint64_t code, int32_t a, int32_t b,
                                  SigStats& st) {
    const bool lead = lane_id() == 0;
    const bool cached = cacheable(c, G, a, b);
    const uint64_t key = sig_key(code, a, b);
    uint32_t v = 0;
    int found = 0;
    if (lead) {
        ++st.lookups;
        if (cached && sig_find(c, key, v)) {
            ++st.hits;
            found = 1;
        }
    }
    found = __shfl_sync(kFull, found, 0);
    if (found) return __shfl_sync(kFull, v, 0);
    v = common_warp(G, a, b);
    if (lead && cached) sig_put(c, key, v);
    return v;
}

// Row of the out-arc a (offp[u] <= a < offp[u + 1]).
__device__ __forceinline__ int32_t arc_source(const int64_t* __restrict__ offp, int64_t n, int64_t a) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (offp[mid] <= a) lo = mid;
        else hi = mid;
    }
    return (int32_t)lo;
}

// Stage C_uv = N(u) n N(v) (sorted) in buf when it has at most kStageCap members; returns |C_uv| in
// every lane and *staged.  x_in_v(x) membership of N(u)'s elements in N(v) by binary search.
__device__ uint32_t stage_common(const Graph& G, int32_t u, int32_t v, int32_t* buf, bool* staged) {
    const int l = lane_id();
    const int64_t ub = G.off[u], ue = G.off[u + 1], vb = G.off[v], ve = G.off[v + 1];
    uint32_t t = 0;
    for (int64_t k0 = ub; k0 < ue; k0 += 32) {
        const int64_t k = k0 + l;
        const int32_t x = k < ue ? __ldg(G.cols + k) : -1;
        const bool in = k < ue && row_has(G.cols, vb, ve, x);
        const uint32_t bal = __ballot_sync(kFull, in);
        const uint32_t pos = t + __popc(bal & lanemask_lt());
        if (in && pos < (uint32_t)kStageCap) buf[pos] = x;
        t += __popc(bal);
    }
    __syncwarp();
    *staged = t <= (uint32_t)kStageCap;
    return t;
}

// 128-bit sums: (lo, hi) words of acc, added with the carry of the low word.
__device__ __forceinline__ void add128(uint64_t* acc_lo, unsigned __int128 v) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    const unsigned long long old = atomicAdd((unsigned long long*)acc_lo, lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd((unsigned long long*)(acc_lo + 1), hi + carry);
}

__device__ __forceinline__ void flush_u64(uint64_t* dst, uint64_t v, uint64_t* red) {
    v = block_sum_u64(v, red);
    if (threadIdx.x == 0 && v) atomicAdd((unsigned long long*)dst, (unsigned long long)v);
}

// per-thread 128-bit partial -> one 128-bit atomic per block (low and high words reduced apart; the
// low words' carries are counted by summing them as 128-bit through two 32-bit halves)
__device__ __forceinline__ void flush_u128(uint64_t* dst_lo, unsigned __int128 v, uint64_t* red) {
    const uint64_t lo32 = (uint64_t)v & 0xffffffffull;
    const uint64_t hi32 = (uint64_t)(v >> 32) & 0xffffffffull;
    const uint64_t top = (uint64_t)(v >> 64);
    const uint64_t s_lo32 = block_sum_u64(lo32, red);  // < 2^32 * threads: no overflow
    const uint64_t s_hi32 = block_sum_u64(hi32, red);
    const uint64_t s_top = block_sum_u64(top, red);
    if (threadIdx.x == 0) {
        const unsigned __int128 total = (unsigned __int128)s_lo32 + ((unsigned __int128)s_hi32 << 32) +
                                        ((unsigned __int128)s_top << 64);
        if (total) add128(dst_lo, total);
    }
}

__device__ __forceinline__ void flush_stats(uint64_t* acc, const SigStats& st, uint64_t* red) {
    flush_u64(&acc[ACC_SIG_LOOKUPS], st.lookups, red);
    flush_u64(&acc[ACC_SIG_HITS], st.hits, red);
}

// ---------------------------------------------------------------------------------------------
// 1. Triangles: X_1, X_2, X_3 per triangle; tau3 per vertex.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kLitThreads) k_lit_tri(Graph G, const int64_t* __restrict__ offp,
                                                         const int32_t* __restrict__ colsp, int64_t n, int64_t m,
                                                         SigCache cache, uint64_t* __restrict__ tau3,
                                                         uint64_t* __restrict__ acc) {
    __shared__ int32_t sbuf[kLitWarps][kStageCap];
    __shared__ uint64_t red[32];
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    SigStats st;
    uint64_t x1 = 0, tri = 0;
    unsigned __int128 x2 = 0, x3 = 0;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < m; a += nw) {
        const int32_t u = arc_source(offp, n, a);
        const int32_t v = colsp[a];
        bool staged = false;
        const uint32_t t_uv = stage_common(G, u, v, sbuf[w], &staged);
        if (l == 0) {  // this arc computed C_uv itself: one request, answered by the computation
            ++st.lookups;
            if (cacheable(cache, G, u, v)) sig_put(cache, sig_key(SIG_C, u, v), t_uv);
        }
        if (t_uv == 0) continue;
        const uint64_t du = (uint64_t)G.deg[u], dv = (uint64_t)G.deg[v];
        const int64_t ub = G.off[u], ue = G.off[u + 1], vb = G.off[v], ve = G.off[v + 1];
        // one triangle (u, v, wv), the whole warp
        auto triangle = [&](int32_t wv) {
            const int64_t wb = G.off[wv], we = G.off[wv + 1];
            uint32_t c3 = 0;  // X_3 = |C_uv n N(w)|
            if (staged) {
                for (uint32_t k = l; k < t_uv; k += 32) c3 += row_has(G.cols, wb, we, sbuf[w][k]) ? 1u : 0u;
            } else {
                for (int64_t k = ub + l; k < ue; k += 32) {
                    const int32_t x = __ldg(G.cols + k);
                    c3 += (row_has(G.cols, vb, ve, x) && row_has(G.cols, wb, we, x)) ? 1u : 0u;
                }
            }
            c3 = warp_sum(c3);
            const uint32_t t_uw = frontier_warp(cache, G, SIG_C, u, wv, st);
            const uint32_t t_vw = frontier_warp(cache, G, SIG_C, v, wv, st);
            if (l == 0) {
                const uint64_t X3 = c3;
                const uint64_t X2 = ((uint64_t)t_uv - 1) + ((uint64_t)t_uw - 1) + ((uint64_t)t_vw - 1) - 3 * X3;
                const uint64_t X1 = (du + dv + (uint64_t)G.deg[wv] - 6) - 2 * X2 - 3 * X3;
                x1 += X1;
                x2 += X2;
                x3 += X3;
                ++tri;
                if (X3) {
                    atomicAdd((unsigned long long*)&tau3[u], (unsigned long long)X3);
                    atomicAdd((unsigned long long*)&tau3[v], (unsigned long long)X3);
                    atomicAdd((unsigned long long*)&tau3[wv], (unsigned long long)X3);
                }
            }
        };
        // the triangles anchored here: w in C_uv above v (C_uv is sorted)
        if (staged) {
            uint32_t below = 0;
            for (uint32_t k = l; k < t_uv; k += 32) below += sbuf[w][k] < v ? 1u : 0u;
            for (uint32_t i = warp_sum(below); i < t_uv; ++i) triangle(sbuf[w][i]);
        } else {  // C_uv did not fit: walk N(u) above v again, 32 elements at a time
            for (int64_t k0 = row_lb(G.cols, ub, ue, v + 1); k0 < ue; k0 += 32) {
                const int64_t k = k0 + l;
                const int32_t x = k < ue ? __ldg(G.cols + k) : -1;
                uint32_t bal = __ballot_sync(kFull, k < ue && row_has(G.cols, vb, ve, x));
                while (bal) {
                    const int src = __ffs(bal) - 1;
                    bal &= bal - 1;
                    triangle(__shfl_sync(kFull, x, src));
                }
            }
        }
        __syncwarp();
    }
    flush_u64(&acc[ACC_LIT_X1], x1, red);
    flush_u64(&acc[ACC_LIT_T], tri, red);
    flush_u128(&acc[ACC_LIT_X2], x2, red);
    flush_u128(&acc[ACC_LIT_X3], x3, red);
    flush_stats(acc, st, red);
}

// ---------------------------------------------------------------------------------------------
// 2. Edges: |A_e| |B_e| and the A_e x B_e pairs that are edges.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kLitThreads) k_lit_edge(Graph G, const int64_t* __restrict__ offp,
                                                          const int32_t* __restrict__ colsp, int64_t n, int64_t m,
                                                          SigCache cache, uint64_t* __restrict__ acc) {
    __shared__ int32_t sbuf[kLitWarps][kStageCap];
    __shared__ uint64_t red[32];
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    SigStats st;
    uint64_t ab_sum = 0;
    unsigned __int128 e_sum = 0;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < m; a += nw) {
        const int32_t u = arc_source(offp, n, a);
        const int32_t v = colsp[a];
        const uint32_t t = frontier_warp(cache, G, SIG_C, u, v, st);
        const uint64_t A = (uint64_t)G.deg[u] - 1 - t, B = (uint64_t)G.deg[v] - 1 - t;
        if (l == 0) ab_sum += A * B;
        if (A == 0 || B == 0) continue;  // no pair
        bool staged = false;
        stage_common(G, u, v, sbuf[w], &staged);
        const int64_t ub = G.off[u], ue = G.off[u + 1], vb = G.off[v], ve = G.off[v + 1];
        uint64_t e_part = 0;
        // x in A_e: the elements of N(u) other than v that are not in N(v), one per lane
        for (int64_t k = ub + l; k < ue; k += 32) {
            const int32_t x = __ldg(G.cols + k);
            if (x == v || row_has(G.cols, vb, ve, x)) continue;
            const uint32_t cxv = frontier_serial(cache, G, SIG_W, x, v, st);  // |N(x) n N(v)|, x !~ v
            const int64_t xb = G.off[x], xe = G.off[x + 1];
            uint32_t cc = 0;  // |C_uv n N(x)|
            if (staged) {
                if ((int64_t)t <= xe - xb) {
                    for (uint32_t q = 0; q < t; ++q) cc += row_has(G.cols, xb, xe, sbuf[w][q]) ? 1u : 0u;
                } else {
                    for (int64_t q = xb; q < xe; ++q) {
                        const int32_t y = __ldg(G.cols + q);
                        int lo = 0, hi = (int)t;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (sbuf[w][mid] < y) lo = mid + 1;
                            else hi = mid;
                        }
                        cc += (lo < (int)t && sbuf[w][lo] == y) ? 1u : 0u;
                    }
                }
            } else {
                for (int64_t q = xb; q < xe; ++q) {
                    const int32_t y = __ldg(G.cols + q);
                    cc += (row_has(G.cols, ub, ue, y) && row_has(G.cols, vb, ve, y)) ? 1u : 0u;
                }
            }
            e_part += (uint64_t)cxv - 1 - cc;  // u is in N(x) n N(v) too
        }
        e_sum += warp_sum(e_part);  // identical in every lane: lane 0 keeps it
        if (l != 0) e_sum = 0;
        __syncwarp();
    }
    flush_u64(&acc[ACC_LIT_AB], ab_sum, red);
    flush_u128(&acc[ACC_LIT_E], e_sum, red);
    flush_stats(acc, st, red);
}

// ---------------------------------------------------------------------------------------------
// 3. Vertices: the star form on H_u.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kLitThreads) k_lit_star(Graph G, int64_t n, SigCache cache,
                                                          const uint64_t* __restrict__ tau3,
                                                          uint64_t* __restrict__ acc) {
    __shared__ uint64_t red[32];
    const int l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    SigStats st;
    uint64_t star = 0, bad = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const int64_t ub = G.off[u], ue = G.off[u + 1];
        uint64_t s1 = 0, s2 = 0;  // sum deg_H(v), sum C(deg_H(v), 2)
        for (int64_t k = ub + l; k < ue; k += 32) {
            const int32_t v = __ldg(G.cols + k);
            const uint64_t t = frontier_serial(cache, G, SIG_C, (int32_t)u, v, st);
            s1 += t;
            s2 += choose2_u64(t);
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if (l == 0) {
            const uint64_t d = (uint64_t)(ue - ub);
            const uint64_t t3 = tau3[u];
            bad |= (s1 & 1) | (t3 % 3 ? 1 : 0);
            const uint64_t mH = s1 >> 1, tau = t3 / 3;
            star += choose3_u64(d) - mH * (d >= 2 ? d - 2 : 0) + s2 - tau;
        }
    }
    flush_u64(&acc[ACC_LIT_STAR], star, red);
    bad = block_sum_u64(bad, red);
    if (threadIdx.x == 0 && bad) atomicOr((unsigned long long*)&acc[ACC_ERR], (unsigned long long)kErrLitDiv);
    flush_stats(acc, st, red);
}

// ---------------------------------------------------------------------------------------------
// 4. The closure as printed, and the non-induced statistics it implies.
// ---------------------------------------------------------------------------------------------
__global__ void k_lit_close(int64_t m, uint64_t* __restrict__ acc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned __int128 X2 = (unsigned __int128)acc[ACC_LIT_X2] | ((unsigned __int128)acc[ACC_LIT_X2 + 1] << 64);
    const unsigned __int128 X3 = (unsigned __int128)acc[ACC_LIT_X3] | ((unsigned __int128)acc[ACC_LIT_X3 + 1] << 64);
    const unsigned __int128 E = (unsigned __int128)acc[ACC_LIT_E] | ((unsigned __int128)acc[ACC_LIT_E + 1] << 64);
    if ((X2 & 1) || (X3 & 3) || (E & 3))
        atomicOr((unsigned long long*)&acc[ACC_ERR], (unsigned long long)kErrLitDiv);
    const uint64_t paw = acc[ACC_LIT_X1];
    const uint64_t diamond = (uint64_t)(X2 >> 1);
    const uint64_t k4 = (uint64_t)(X3 >> 2);
    const uint64_t cycle = (uint64_t)(E >> 2);
    const uint64_t path = acc[ACC_LIT_AB] - (uint64_t)E;
    const uint64_t star = acc[ACC_LIT_STAR];
    acc[OUT_COUNTS + HARP_STAR3] = star;
    acc[OUT_COUNTS + HARP_PATH4] = path;
    acc[OUT_COUNTS + HARP_PAW] = paw;
    acc[OUT_COUNTS + HARP_CYCLE4] = cycle;
    acc[OUT_COUNTS + HARP_DIAMOND] = diamond;
    acc[OUT_COUNTS + HARP_CLIQUE4] = k4;
    // the non-induced statistics, by the containment of each pattern in the induced classes (the
    // forward direction of the system the triangle-wedge basis inverts); T as enumerated
    acc[OUT_STATS + HARP_STAT_TRIANGLES] = acc[ACC_LIT_T];
    acc[OUT_STATS + HARP_STAT_K4] = k4;
    acc[OUT_STATS + HARP_STAT_C4] = cycle + diamond + 3 * k4;
    acc[OUT_STATS + HARP_STAT_STARS] = star + paw + 2 * diamond + 4 * k4;
    acc[OUT_STATS + HARP_STAT_PATHS] = path + 2 * paw + 4 * cycle + 6 * diamond + 12 * k4;
    acc[OUT_STATS + HARP_STAT_PAWS] = paw + 4 * diamond + 12 * k4;
    acc[OUT_STATS + HARP_STAT_DIAMONDS] = diamond + 6 * k4;
    acc[OUT_STATS + HARP_STAT_EDGES] = (uint64_t)m;
}

unsigned lit_grid(int64_t warps) {
    int64_t b = (warps * 32 + kLitThreads - 1) / kLitThreads;
    if (b < 1) b = 1;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)(b > cap ? cap : b);
}

}  // namespace

harp_status count_literal(const harp_csr* g, Workspace& ws, const harp_plan& plan, cudaStream_t s) {
    const int64_t n = g->n, m = g->m;
    // cache slots: 2^lit_cache_log2, or the power of two >= 4m (at most 2^25); off with NO_REUSE
    const bool use_cache = !(plan.flags & HARP_PLAN_NO_REUSE) && m > 0;
    int lg = (int)plan.lit_cache_log2;
    if (lg == 0) {
        lg = 10;
        while (lg < 25 && ((int64_t)1 << lg) < 4 * m) ++lg;
    }
    const size_t slots = use_cache ? ((size_t)1 << lg) : 0;
    const size_t bytes = 16 * slots + 8 * (size_t)(n > 0 ? n : 1);
    unsigned char* scratch = nullptr;
    HARP_CK(cudaMallocAsync((void**)&scratch, bytes, s));
    SigCache cache{nullptr, nullptr, 0, (int32_t)plan.lit_cache_min_deg};
    if (slots) {
        cache.keys = reinterpret_cast<unsigned long long*>(scratch);
        cache.vals = cache.keys + slots;
        cache.mask = (uint32_t)(slots - 1);
    }
    uint64_t* tau3 = reinterpret_cast<uint64_t*>(scratch + 16 * slots);
    const Graph G{ws.off, ws.cols, ws.deg};
    cudaError_t e = cudaSuccess;
    if (slots) e = cudaMemsetAsync(cache.keys, 0xff, 8 * slots, s);
    if (e == cudaSuccess && slots) e = cudaMemsetAsync(cache.vals, 0, 8 * slots, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tau3, 0, 8 * (size_t)(n > 0 ? n : 1), s);
    if (e == cudaSuccess && m > 0) {
        k_lit_tri<<<lit_grid(m), kLitThreads, 0, s>>>(G, ws.offp, ws.colsp, n, m, cache, tau3, ws.acc);
        note_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = prof_mark(s, SEG_TRI_WARP);
        if (e == cudaSuccess) {
            k_lit_edge<<<lit_grid(m), kLitThreads, 0, s>>>(G, ws.offp, ws.colsp, n, m, cache, ws.acc);
            note_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = prof_mark(s, SEG_C4_SMALL);
        if (e == cudaSuccess) {
            k_lit_star<<<lit_grid(n), kLitThreads, 0, s>>>(G, n, cache, tau3, ws.acc);
            note_launch();
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        k_lit_close<<<1, 32, 0, s>>>(m, ws.acc);
        note_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return HARP_ECUDA;
    }
    return HARP_OK;
}

}  // namespace harp
