// Per-vertex (orbit) counts of the connected induced 4-vertex motifs: an output mode beside the
// global counts of Section III-F (the paper's closure is global; this refines every induced
// occurrence S by the role of each of its vertices, the role being the vertex's automorphism class
// in the motif, which for 4-vertex motifs its degree inside G[S] decides).  Eleven roles, in order:
//   0 star centre  1 star leaf  2 path end  3 path inner  4 paw pendant  5 paw hub (degree 3)
//   6 paw side (degree-2 triangle vertex)  7 cycle  8 diamond spine (degree 3)  9 diamond tip
//   10 clique
// The same closure idea as the global counts, per vertex: eleven non-induced statistics N_i(v) (copies
// of a pattern in which v plays role i) are sums of degrees, per-edge triangle counts t_e, per-vertex
// triangle, 4-cycle and 4-clique counts, and their containment in the induced roles is a unit
// upper-triangular integer matrix, so the roles follow by back-substitution without division:
//   N0 = C(d_v, 3)                                N1 = sum_{c in N(v)} C(d_c - 1, 2)
//   N2 = sum_{a in N(v)} S1(a) - d_v (d_v - 1) - 2 t_v,  S1(a) = sum_{b in N(a)} (d_b - 1)
//   N3 = (d_v - 1) S1(v) - 2 t_v                  N4 = sum_{h in N(v)} t_h - 2 t_v
//   N5 = t_v (d_v - 2)                            N6 = sum_{h in N(v)} t_vh (d_h - 2)
//   N7 = 4-cycles through v                       N8 = sum_{s in N(v)} C(t_vs, 2)
//   N9 = sum over triangles {v, a, b} of (t_ab - 1)
//   N10 = 4-cliques through v = tau(H_v) = (1/3) sum over triangles T on v of X_3(T)
// with t_v = (1/2) sum_{h in N(v)} t_vh the triangles on v.
//
// Passes after orientation and the triangle pass (which leaves t_e of every out-arc in ws.te):
//   k_orb_tri     warp per out-arc (u, v): the frontier C_uv = N(u) n N(v), staged; every triangle
//                 (u, v, w), w in C_uv above v, routes t_vw - 1, t_uw - 1, t_uv - 1 to N9 of u, v, w
//                 and X_3 = |C_uv n N(w)| to tau3 of all three
//   k_orb_vertex  warp per vertex: t_v, S1(v), N1, N6, N8
//   k_orb_c4w     warp per root u with wedge work W(u) <= kHashMax (a shared-memory hash), and
//   k_orb_c4b     a block per heavier root (dense counters over all ranks in a per-block global
//                 array): every 4-cycle has one top vertex u, opposite corner x and middles w1, w2
//                 below u; with cnt(x) the wedges u - w - x, u gets sum_x C(cnt(x), 2), x gets
//                 C(cnt(x), 2) (as half of sum over its wedges of cnt(x) - 1) and each middle w gets
//                 sum_{x in its segment} (cnt(x) - 1)
//   k_orb_close   warp per vertex: N2, N4, N0, N3, N5, N9, N10 and the back-substitution, written to
//                 the input id of the vertex.
//
// Per-edge (edge orbit) counts use the same passes with routing to edges instead of vertices: ten
// roles of an edge inside G[S] (its endpoints' degrees there decide them), ten statistics E_i(e) for
// e = (a, b) and a unit upper-triangular 10 x 10 containment system:
//   E0 = C(d_a - 1, 2) + C(d_b - 1, 2)          E1 = S1(a) + S1(b) - d_a - d_b + 2 - 2 t_ab
//   E2 = (d_a - 1)(d_b - 1) - t_ab              E3 = t_a + t_b - 2 t_ab
//   E4 = t_ab (d_a + d_b - 4)                   E5 = sum_{h in N(a) n N(b)} (d_h - 2)
//   E6 = 4-cycles through e                     E7 = C(t_ab, 2)
//   E8 = sum_{s in N(a) n N(b)} (t_as - 1) + (t_bs - 1)
//   E9 = 4-cliques through e = (1/2) sum over the triangles T on e of X_3(T)
// E5, E8 and E9 are routed from each triangle to its three edges (k_orb_tri), E6 from the wedge walk:
// each wedge u - w - x adds cnt(x) - 1 to the arcs (u, w) and (w, x) (k_orb_c4w / k_orb_c4b), and
// k_eorb_close evaluates one edge per thread and writes it at the edge's index in the input graph's
// edge list ((a, b), a < b, lexicographic by input id).
#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kOrbThreads = 256;
constexpr int kOrbWarps = kOrbThreads / 32;
constexpr int kOrbStage = 512;      // C_uv members staged per warp
constexpr int kHashSlots = 1024;    // per-warp wedge hash (roots with W(u) <= kHashMax)
constexpr int kHashMax = 512;
constexpr int32_t kNoKey = -1;
constexpr int kOrbits = 11;

// the containment matrix of the per-vertex system (row: statistic, column: role), unit upper triangular
__constant__ uint8_t c_contain[kOrbits][kOrbits] = {
    {1, 0, 0, 0, 0, 1, 0, 0, 1, 0, 1}, {0, 1, 0, 0, 1, 0, 1, 0, 1, 2, 3}, {0, 0, 1, 0, 2, 0, 1, 2, 2, 4, 6},
    {0, 0, 0, 1, 0, 2, 1, 2, 4, 2, 6}, {0, 0, 0, 0, 1, 0, 0, 0, 0, 2, 3}, {0, 0, 0, 0, 0, 1, 0, 0, 2, 0, 3},
    {0, 0, 0, 0, 0, 0, 1, 0, 2, 2, 6}, {0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 3}, {0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 3},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 3}, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1}};

struct OrbGraph {
    const int64_t* off;    // rank-order CSR, rows sorted
    const int32_t* cols;
    const int32_t* deg;
    const int64_t* offp;   // out-lists N+(v) and t_e of every out-arc
    const int32_t* colsp;
    const uint32_t* te;
};

__device__ __forceinline__ bool has(const int32_t* __restrict__ cols, int64_t b, int64_t e, int32_t x) {
    const int64_t p = b + lower_bound_i32(cols + b, e - b, x);
    return p < e && __ldg(cols + p) == x;
}

// the out-arc of the edge {a, b} (a != b adjacent): the lower rank's out-list holds the higher one
__device__ __forceinline__ int64_t arc_of(const OrbGraph& G, int32_t a, int32_t b) {
    const int32_t lo = a < b ? a : b, hi = a < b ? b : a;
    const int64_t pb = G.offp[lo], pe = G.offp[lo + 1];
    return pb + lower_bound_i32(G.colsp + pb, pe - pb, hi);
}
// t of the edge {a, b}
__device__ __forceinline__ uint64_t t_of(const OrbGraph& G, int32_t a, int32_t b) {
    return (uint64_t)G.te[arc_of(G, a, b)];
}

__device__ __forceinline__ int32_t arc_row(const int64_t* __restrict__ offp, int64_t n, int64_t a) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (offp[mid] <= a) lo = mid;
        else hi = mid;
    }
    return (int32_t)lo;
}

// ---------------------------------------------------------------------------------------------
// Triangles: N9 and tau3 routing.
// ---------------------------------------------------------------------------------------------
// Per-edge routing targets of the triangle pass (per out-arc; all nullptr for the per-vertex mode).
struct EdgeRoute {
    unsigned long long* e5;  // sum of (d of the third vertex - 2)
    unsigned long long* e8;  // sum of (t - 1) of the other two edges
    unsigned long long* e9;  // sum of X_3 (twice the 4-cliques through the edge)
};

__global__ void __launch_bounds__(kOrbThreads) k_orb_tri(OrbGraph G, int64_t n, int64_t m,
                                                         unsigned long long* __restrict__ n9,
                                                         unsigned long long* __restrict__ tau3, EdgeRoute er) {
    __shared__ int32_t sbuf[kOrbWarps][kOrbStage];
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < m; a += nw) {
        const int32_t u = arc_row(G.offp, n, a);
        const int32_t v = G.colsp[a];
        const uint64_t t_uv = G.te[a];
        if (t_uv == 0) continue;
        const int64_t ub = G.off[u], ue = G.off[u + 1], vb = G.off[v], ve = G.off[v + 1];
        const bool staged = t_uv <= (uint64_t)kOrbStage;
        if (staged) {  // C_uv in rank order
            uint32_t t = 0;
            for (int64_t k0 = ub; k0 < ue; k0 += 32) {
                const int64_t k = k0 + l;
                const int32_t x = k < ue ? __ldg(G.cols + k) : -1;
                const bool in = k < ue && has(G.cols, vb, ve, x);
                const uint32_t bal = __ballot_sync(kFull, in);
                const uint32_t pos = t + __popc(bal & lanemask_lt());
                if (in && pos < (uint32_t)kOrbStage) sbuf[w][pos] = x;  // pos < t_uv <= kOrbStage
                t += __popc(bal);
            }
            __syncwarp();
        }
        auto triangle = [&](int32_t wv) {
            const int64_t wb = G.off[wv], we = G.off[wv + 1];
            uint32_t c3 = 0;
            if (staged) {
                for (uint32_t k = l; k < t_uv; k += 32) c3 += has(G.cols, wb, we, sbuf[w][k]) ? 1u : 0u;
            } else {
                for (int64_t k = ub + l; k < ue; k += 32) {
                    const int32_t x = __ldg(G.cols + k);
                    c3 += (has(G.cols, vb, ve, x) && has(G.cols, wb, we, x)) ? 1u : 0u;
                }
            }
            c3 = warp_sum(c3);
            if (l == 0 && n9) {
                const uint64_t t_uw = t_of(G, u, wv), t_vw = t_of(G, v, wv);
                atomicAdd(&n9[u], (unsigned long long)(t_vw - 1));
                atomicAdd(&n9[v], (unsigned long long)(t_uw - 1));
                atomicAdd(&n9[wv], (unsigned long long)(t_uv - 1));
                if (c3) {
                    atomicAdd(&tau3[u], (unsigned long long)c3);
                    atomicAdd(&tau3[v], (unsigned long long)c3);
                    atomicAdd(&tau3[wv], (unsigned long long)c3);
                }
            }
            if (l == 0 && er.e5) {  // the triangle's three edges: (u, v) = arc a, (u, w), (v, w)
                const int64_t a_uw = arc_of(G, u, wv), a_vw = arc_of(G, v, wv);
                const uint64_t t_uw = G.te[a_uw], t_vw = G.te[a_vw];
                const uint64_t du = (uint64_t)G.deg[u], dv = (uint64_t)G.deg[v], dw = (uint64_t)G.deg[wv];
                atomicAdd(&er.e5[a], (unsigned long long)(dw - 2));
                atomicAdd(&er.e5[a_uw], (unsigned long long)(dv - 2));
                atomicAdd(&er.e5[a_vw], (unsigned long long)(du - 2));
                atomicAdd(&er.e8[a], (unsigned long long)((t_uw - 1) + (t_vw - 1)));
                atomicAdd(&er.e8[a_uw], (unsigned long long)((t_uv - 1) + (t_vw - 1)));
                atomicAdd(&er.e8[a_vw], (unsigned long long)((t_uv - 1) + (t_uw - 1)));
                if (c3) {
                    atomicAdd(&er.e9[a], (unsigned long long)c3);
                    atomicAdd(&er.e9[a_uw], (unsigned long long)c3);
                    atomicAdd(&er.e9[a_vw], (unsigned long long)c3);
                }
            }
        };
        if (staged) {
            uint32_t below = 0;
            for (uint32_t k = l; k < t_uv; k += 32) below += sbuf[w][k] < v ? 1u : 0u;
            for (uint32_t i = warp_sum(below); i < t_uv; ++i) triangle(sbuf[w][i]);
        } else {
            for (int64_t k0 = ub + lower_bound_i32(G.cols + ub, ue - ub, v + 1); k0 < ue; k0 += 32) {
                const int64_t k = k0 + l;
                const int32_t x = k < ue ? __ldg(G.cols + k) : -1;
                uint32_t bal = __ballot_sync(kFull, k < ue && has(G.cols, vb, ve, x));
                while (bal) {
                    const int src = __ffs(bal) - 1;
                    bal &= bal - 1;
                    triangle(__shfl_sync(kFull, x, src));
                }
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------------
// Per-vertex sums over the neighbourhood.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kOrbThreads) k_orb_vertex(OrbGraph G, int64_t n, uint64_t* __restrict__ tsum,
                                                            uint64_t* __restrict__ s1, uint64_t* __restrict__ N) {
    const int l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const int64_t vb = G.off[v], ve = G.off[v + 1];
        uint64_t ts = 0, sa = 0, n1 = 0, n6 = 0, n8 = 0;
        for (int64_t k = vb + l; k < ve; k += 32) {
            const int32_t h = __ldg(G.cols + k);
            const uint64_t dh = (uint64_t)G.deg[h];
            const uint64_t t = t_of(G, (int32_t)v, h);
            ts += t;
            sa += dh - 1;
            n1 += choose2_u64(dh - 1);
            n6 += t * (dh - 2);  // dh >= 2 whenever t > 0
            n8 += choose2_u64(t);
        }
        ts = warp_sum(ts);
        sa = warp_sum(sa);
        n1 = warp_sum(n1);
        n6 = warp_sum(n6);
        n8 = warp_sum(n8);
        if (l == 0) {
            tsum[v] = ts;
            s1[v] = sa;
            N[v * kOrbits + 1] = n1;
            N[v * kOrbits + 6] = n6;
            N[v * kOrbits + 8] = n8;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// 4-cycles through each vertex (N7), by the wedge anchor with per-role routing.
// ---------------------------------------------------------------------------------------------
// Wedge work of root u: sum over w in N-(u) of |{x in N(w) : x < u}| (x = u excluded: it is the
// position of u in w's row).  Light roots are queued for the warp kernel, the rest for the block one.
__global__ void k_orb_classify(OrbGraph G, int64_t n, int32_t* __restrict__ q_light, int32_t* __restrict__ q_heavy,
                               unsigned long long* __restrict__ qcnt) {
    const int l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const int64_t ub = G.off[u];
        const int64_t dm = (int64_t)G.deg[u] - (G.offp[u + 1] - G.offp[u]);  // |N-(u)|
        if (dm < 2) continue;
        uint64_t W = 0;
        for (int64_t k = l; k < dm; k += 32) {
            const int32_t w = __ldg(G.cols + ub + k);
            const int64_t wb = G.off[w];
            W += (uint64_t)lower_bound_i32(G.cols + wb, G.off[w + 1] - wb, (int32_t)u);
        }
        W = warp_sum(W);
        if (l == 0 && W > 0) {
            if (W <= (uint64_t)kHashMax) q_light[atomicAdd(&qcnt[0], 1ull)] = (int32_t)u;
            else q_heavy[atomicAdd(&qcnt[1], 1ull)] = (int32_t)u;
        }
    }
}

__device__ __forceinline__ uint32_t* hash_slot(int32_t* keys, uint32_t* cnt, int32_t x, bool insert) {
    uint32_t h = hash32((uint32_t)x) & (kHashSlots - 1);
    for (;;) {
        int32_t k = keys[h];
        if (k == kNoKey) {
            if (!insert) return nullptr;
            const int32_t prev = atomicCAS(&keys[h], kNoKey, x);
            if (prev == kNoKey || prev == x) return &cnt[h];
            k = prev;
        }
        if (k == x) return &cnt[h];
        h = (h + 1) & (kHashSlots - 1);
    }
}

__global__ void __launch_bounds__(kOrbThreads) k_orb_c4w(OrbGraph G, const int32_t* __restrict__ q,
                                                         const unsigned long long* __restrict__ qcnt,
                                                         unsigned long long* __restrict__ n7,
                                                         unsigned long long* __restrict__ n7x2,
                                                         unsigned long long* __restrict__ e6a) {
    __shared__ int32_t keys[kOrbWarps][kHashSlots];
    __shared__ uint32_t cnt[kOrbWarps][kHashSlots];
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nq = (int64_t)qcnt[0];
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nq; i += nw) {
        const int32_t u = q[i];
        for (int k = l; k < kHashSlots; k += 32) {
            keys[w][k] = kNoKey;
            cnt[w][k] = 0;
        }
        __syncwarp();
        const int64_t ub = G.off[u];
        const int64_t dm = (int64_t)G.deg[u] - (G.offp[u + 1] - G.offp[u]);
        // pass 1: cnt(x) over the wedges u - w - x, x < u (a lane per lower neighbour)
        for (int64_t k = l; k < dm; k += 32) {
            const int32_t wv = __ldg(G.cols + ub + k);
            const int64_t wb = G.off[wv];
            const int64_t we = wb + lower_bound_i32(G.cols + wb, G.off[wv + 1] - wb, u);
            for (int64_t p = wb; p < we; ++p) atomicAdd(hash_slot(keys[w], cnt[w], __ldg(G.cols + p), true), 1u);
        }
        __syncwarp();
        // pass 2: each middle w gets sum (cnt(x) - 1) over its segment; each occurrence of x adds
        // cnt(x) - 1 to x's doubled count; the root gets half the total
        uint64_t root2 = 0;
        for (int64_t k = l; k < dm; k += 32) {
            const int32_t wv = __ldg(G.cols + ub + k);
            const int64_t wb = G.off[wv];
            const int64_t we = wb + lower_bound_i32(G.cols + wb, G.off[wv + 1] - wb, u);
            uint64_t sw = 0;
            for (int64_t p = wb; p < we; ++p) {
                const int32_t x = __ldg(G.cols + p);
                const uint32_t c = *hash_slot(keys[w], cnt[w], x, false) - 1u;
                sw += c;
                if (c && n7x2) atomicAdd(&n7x2[x], (unsigned long long)c);
                if (c && e6a) atomicAdd(&e6a[p], (unsigned long long)c);  // the arc (w, x)
            }
            if (sw && n7) atomicAdd(&n7[wv], (unsigned long long)sw);
            if (sw && e6a) atomicAdd(&e6a[ub + k], (unsigned long long)sw);  // the arc (u, w)
            root2 += sw;
        }
        root2 = warp_sum(root2);
        if (l == 0 && root2 && n7) atomicAdd(&n7[u], (unsigned long long)(root2 >> 1));
        __syncwarp();
    }
}

// Heavy roots: one block each (persistent blocks over the queue), dense counters over every rank in
// the block's slice of a global array (cleared again by a third walk).
__global__ void __launch_bounds__(kOrbThreads) k_orb_c4b(OrbGraph G, int64_t n, const int32_t* __restrict__ q,
                                                         const unsigned long long* __restrict__ qcnt,
                                                         uint32_t* __restrict__ dense,
                                                         unsigned long long* __restrict__ n7,
                                                         unsigned long long* __restrict__ n7x2,
                                                         unsigned long long* __restrict__ e6a) {
    __shared__ uint64_t red[32];
    uint32_t* cntv = dense + (size_t)blockIdx.x * (size_t)n;
    const int64_t nq = (int64_t)qcnt[1];
    const int w = threadIdx.x >> 5, l = lane_id();
    for (int64_t i = blockIdx.x; i < nq; i += gridDim.x) {
        const int32_t u = q[i];
        const int64_t ub = G.off[u];
        const int64_t dm = (int64_t)G.deg[u] - (G.offp[u + 1] - G.offp[u]);
        // warp per lower neighbour, lanes along its segment
        for (int pass = 0; pass < 3; ++pass) {
            uint64_t root2 = 0;
            for (int64_t k = w; k < dm; k += kOrbWarps) {
                const int32_t wv = __ldg(G.cols + ub + k);
                const int64_t wb = G.off[wv];
                const int64_t we = wb + lower_bound_i32(G.cols + wb, G.off[wv + 1] - wb, u);
                uint64_t sw = 0;
                for (int64_t p = wb + l; p < we; p += 32) {
                    const int32_t x = __ldg(G.cols + p);
                    if (pass == 0) {
                        atomicAdd(&cntv[x], 1u);
                    } else if (pass == 1) {
                        const uint32_t c = cntv[x] - 1u;
                        sw += c;
                        if (c && n7x2) atomicAdd(&n7x2[x], (unsigned long long)c);
                        if (c && e6a) atomicAdd(&e6a[p], (unsigned long long)c);  // the arc (w, x)
                    } else {
                        cntv[x] = 0;
                    }
                }
                if (pass == 1) {
                    sw = warp_sum(sw);
                    if (l == 0 && sw && n7) atomicAdd(&n7[wv], (unsigned long long)sw);
                    if (l == 0 && sw && e6a) atomicAdd(&e6a[ub + k], (unsigned long long)sw);  // the arc (u, w)
                    root2 += sw;
                }
            }
            __syncthreads();  // every counter of the pass is final before the next reads it
            if (pass == 1) {
                root2 = block_sum_u64(l == 0 ? root2 : 0, red);
                if (threadIdx.x == 0 && root2 && n7) atomicAdd(&n7[u], (unsigned long long)(root2 >> 1));
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// The remaining statistics and the back-substitution.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kOrbThreads) k_orb_close(OrbGraph G, int64_t n, const uint64_t* __restrict__ tsum,
                                                           const uint64_t* __restrict__ s1,
                                                           const unsigned long long* __restrict__ n9,
                                                           const unsigned long long* __restrict__ tau3,
                                                           const unsigned long long* __restrict__ n7,
                                                           const unsigned long long* __restrict__ n7x2,
                                                           const int32_t* __restrict__ order,
                                                           uint64_t* __restrict__ N, uint64_t* __restrict__ out,
                                                           uint64_t* __restrict__ acc) {
    const int l = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const int64_t vb = G.off[v], ve = G.off[v + 1];
        uint64_t sa = 0, st = 0;  // sum of S1 and of t_h over the neighbours
        for (int64_t k = vb + l; k < ve; k += 32) {
            const int32_t h = __ldg(G.cols + k);
            sa += s1[h];
            st += tsum[h];
        }
        sa = warp_sum(sa);
        st = warp_sum(st);
        if (l != 0) continue;
        const uint64_t d = (uint64_t)(ve - vb);
        const uint64_t ts = tsum[v];       // 2 t_v
        const uint64_t tv = ts >> 1;
        uint64_t* Nv = N + v * kOrbits;
        uint64_t S[kOrbits];
        S[0] = choose3_u64(d);
        S[1] = Nv[1];
        S[2] = sa - d * (d - 1) - ts;      // sum_a S1(a) - d (d - 1) - 2 t_v
        S[3] = (d - 1) * s1[v] - ts;       // d >= 1 whenever v has a neighbour
        S[4] = (st >> 1) - ts;             // sum_h t_h - 2 t_v (every tsum is even)
        S[5] = tv * (d >= 2 ? d - 2 : 0);
        S[6] = Nv[6];
        S[7] = n7[v] + (n7x2[v] >> 1);
        S[8] = Nv[8];
        S[9] = n9[v];
        S[10] = tau3[v] / 3;
        if ((ts & 1) || (tau3[v] % 3) || (n7x2[v] & 1))
            atomicOr((unsigned long long*)&acc[ACC_ERR], (unsigned long long)kErrLitDiv);
        uint64_t o[kOrbits];
#pragma unroll
        for (int i = kOrbits - 1; i >= 0; --i) {
            uint64_t x = S[i];
#pragma unroll
            for (int j = i + 1; j < kOrbits; ++j) x -= (uint64_t)c_contain[i][j] * o[j];
            o[i] = x;
        }
        uint64_t* dst = out + (int64_t)order[v] * kOrbits;
#pragma unroll
        for (int i = 0; i < kOrbits; ++i) dst[i] = o[i];
    }
}

// ---------------------------------------------------------------------------------------------
// Per-edge statistics and back-substitution.
// ---------------------------------------------------------------------------------------------
constexpr int kEdgeOrbits = 10;
__constant__ uint8_t c_econtain[kEdgeOrbits][kEdgeOrbits] = {
    {1, 0, 0, 1, 1, 0, 0, 2, 1, 2}, {0, 1, 0, 2, 0, 2, 2, 0, 3, 4}, {0, 0, 1, 0, 1, 0, 1, 2, 1, 2},
    {0, 0, 0, 1, 0, 0, 0, 0, 1, 2}, {0, 0, 0, 0, 1, 0, 0, 4, 1, 4}, {0, 0, 0, 0, 0, 1, 0, 0, 1, 2},
    {0, 0, 0, 0, 0, 0, 1, 0, 1, 2}, {0, 0, 0, 0, 0, 0, 0, 1, 0, 1}, {0, 0, 0, 0, 0, 0, 0, 0, 1, 4},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 1}};

// up[x] = neighbours of input vertex x above x (its row's suffix in the input CSR)
__global__ void k_eorb_up(const int64_t* __restrict__ off_in, const int32_t* __restrict__ cols_in, int64_t n,
                          int32_t* __restrict__ up) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = off_in[x], e = off_in[x + 1];
        up[x] = (int32_t)(e - b - lower_bound_i32(cols_in + b, e - b, (int32_t)x + 1));
    }
}

// One thread per out-arc (u, v) of the rank-order graph: the ten statistics, the back-substitution,
// and the write at the edge's index in the input edge list.
__global__ void k_eorb_close(OrbGraph G, int64_t n, int64_t m, const int32_t* __restrict__ dplus,
                             const uint64_t* __restrict__ tsum, const uint64_t* __restrict__ s1,
                             const unsigned long long* __restrict__ e5, const unsigned long long* __restrict__ e8,
                             const unsigned long long* __restrict__ e9, const unsigned long long* __restrict__ e6a,
                             const int32_t* __restrict__ order, const int64_t* __restrict__ off_in,
                             const int32_t* __restrict__ cols_in, const int32_t* __restrict__ up,
                             const int64_t* __restrict__ ebase, uint64_t* __restrict__ out,
                             uint64_t* __restrict__ acc) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = arc_row(G.offp, n, a);
        const int32_t v = G.colsp[a];
        const uint64_t du = (uint64_t)G.deg[u], dv = (uint64_t)G.deg[v];
        const uint64_t t = (uint64_t)G.te[a];
        const uint64_t tu = tsum[u] >> 1, tv = tsum[v] >> 1;
        // the two arcs of the edge in the rank-order CSR: (u, v) in u's suffix, (v, u) in v's prefix
        const int64_t p_uv = G.off[u] + ((int64_t)G.deg[u] - dplus[u]) + (a - G.offp[u]);
        const int64_t vb = G.off[v];
        const int64_t p_vu = vb + lower_bound_i32(G.cols + vb, (int64_t)G.deg[v] - dplus[v], u);
        uint64_t E[kEdgeOrbits];
        E[0] = choose2_u64(du - 1) + choose2_u64(dv - 1);
        E[1] = s1[u] + s1[v] - du - dv + 2 - 2 * t;
        E[2] = (du - 1) * (dv - 1) - t;
        E[3] = tu + tv - 2 * t;
        E[4] = t * (du + dv - 4);
        E[5] = e5[a];
        E[6] = e6a[p_uv] + e6a[p_vu];
        E[7] = choose2_u64(t);
        E[8] = e8[a];
        E[9] = e9[a] >> 1;
        if (e9[a] & 1) atomicOr((unsigned long long*)&acc[ACC_ERR], (unsigned long long)kErrLitDiv);
        uint64_t o[kEdgeOrbits];
#pragma unroll
        for (int i = kEdgeOrbits - 1; i >= 0; --i) {
            uint64_t x = E[i];
#pragma unroll
            for (int j = i + 1; j < kEdgeOrbits; ++j) x -= (uint64_t)c_econtain[i][j] * o[j];
            o[i] = x;
        }
        // index of the edge in the input edge list: (lo, hi) by input id, rows' upper suffixes in order
        const int32_t ia = order[u], ib = order[v];
        const int32_t lo = ia < ib ? ia : ib, hi = ia < ib ? ib : ia;
        const int64_t rb = off_in[lo], re = off_in[lo + 1];
        const int64_t pos = lower_bound_i32(cols_in + rb, re - rb, hi);  // within lo's row
        const int64_t idx = ebase[lo] + (pos - ((re - rb) - up[lo]));
        uint64_t* dst = out + idx * kEdgeOrbits;
#pragma unroll
        for (int i = 0; i < kEdgeOrbits; ++i) dst[i] = o[i];
    }
}

unsigned orb_grid(int64_t warps) {
    int64_t b = (warps * 32 + kOrbThreads - 1) / kOrbThreads;
    if (b < 1) b = 1;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)(b > cap ? cap : b);
}

}  // namespace

harp_status count_orbits(const harp_csr* g, Workspace& ws, uint64_t* d_out, cudaStream_t s) {
    const int64_t n = g->n, m = g->m;
    if (n == 0) return HARP_OK;
    // per-vertex scratch: tsum, s1 (uint64), n9, tau3, n7, n7x2 (uint64), N (11 uint64), two root queues
    // (int32) and their counters; the heavy roots' dense counters (n uint32 per block)
    const size_t per = 6 * 8 + kOrbits * 8 + 2 * 4;
    // heavy roots' dense counters: n uint32 per block, at most 4 GiB in all
    int64_t hb = ((int64_t)4 << 30) / (4 * (n > 0 ? n : 1));
    if (hb > num_sms()) hb = num_sms();
    const int heavy_blocks = hb < 1 ? 1 : (int)hb;
    const size_t dense_bytes = (size_t)heavy_blocks * (size_t)n * 4;
    const size_t bytes = per * (size_t)n + 64 + dense_bytes;
    unsigned char* base = nullptr;
    HARP_CK(cudaMallocAsync((void**)&base, bytes, s));
    uint64_t* tsum = reinterpret_cast<uint64_t*>(base);
    uint64_t* s1 = tsum + n;
    unsigned long long* n9 = reinterpret_cast<unsigned long long*>(s1 + n);
    unsigned long long* tau3 = n9 + n;
    unsigned long long* n7 = tau3 + n;
    unsigned long long* n7x2 = n7 + n;
    uint64_t* N = reinterpret_cast<uint64_t*>(n7x2 + n);
    int32_t* q_light = reinterpret_cast<int32_t*>(N + kOrbits * n);
    int32_t* q_heavy = q_light + n;
    // the two queues hold 2n int32 = 8n bytes, so the counters after them stay 8-byte aligned
    unsigned long long* qcnt = reinterpret_cast<unsigned long long*>(q_heavy + n);
    uint32_t* dense = reinterpret_cast<uint32_t*>(qcnt + 8);
    const OrbGraph G{ws.off, ws.cols, ws.deg, ws.offp, ws.colsp, ws.te};
    cudaError_t e = cudaMemsetAsync(base, 0, bytes, s);  // every accumulator and the dense counters
    auto launched = [&]() {
        note_launch();
        if (e == cudaSuccess) e = cudaGetLastError();
    };
    if (e == cudaSuccess && m > 0) {
        k_orb_tri<<<orb_grid(m), kOrbThreads, 0, s>>>(G, n, m, n9, tau3, EdgeRoute{nullptr, nullptr, nullptr});
        launched();
    }
    if (e == cudaSuccess) {
        k_orb_vertex<<<orb_grid(n), kOrbThreads, 0, s>>>(G, n, tsum, s1, N);
        launched();
    }
    if (e == cudaSuccess && m > 0) {
        k_orb_classify<<<orb_grid(n), kOrbThreads, 0, s>>>(G, n, q_light, q_heavy, qcnt);
        launched();
        if (e == cudaSuccess) {
            k_orb_c4w<<<orb_grid(n), kOrbThreads, 0, s>>>(G, q_light, qcnt, n7, n7x2, nullptr);
            launched();
        }
        if (e == cudaSuccess) {
            k_orb_c4b<<<heavy_blocks, kOrbThreads, 0, s>>>(G, n, q_heavy, qcnt, dense, n7, n7x2, nullptr);
            launched();
        }
    }
    if (e == cudaSuccess) {
        k_orb_close<<<orb_grid(n), kOrbThreads, 0, s>>>(G, n, tsum, s1, n9, tau3, n7, n7x2, ws.order, N, d_out,
                                                         ws.acc);
        launched();
    }
    cudaFreeAsync(base, s);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
    }
    return HARP_OK;
}

}  // namespace harp

namespace harp {

harp_status count_edge_orbits(const harp_csr* g, Workspace& ws, uint64_t* d_out, cudaStream_t s) {
    const int64_t n = g->n, m = g->m;
    if (m == 0) return HARP_OK;
    // scratch: tsum, s1 (uint64 n), N (unused here, 11 n), e5, e8, e9 (uint64 m), e6a (uint64 2m),
    // up (int32 n), ebase (int64 n + 1), root queues (int32 2n), counters, dense counters
    int64_t hb = ((int64_t)4 << 30) / (4 * (n > 0 ? n : 1));
    if (hb > num_sms()) hb = num_sms();
    const int heavy_blocks = hb < 1 ? 1 : (int)hb;
    const size_t bytes = 8 * (size_t)(2 * n) + 8 * (size_t)(11 * n) + 8 * (size_t)(3 * m) + 8 * (size_t)(2 * m) +
                         4 * (size_t)n + 8 * (size_t)(n + 2) + 4 * (size_t)(2 * n) + 128 +
                         (size_t)heavy_blocks * (size_t)n * 4;
    unsigned char* base = nullptr;
    HARP_CK(cudaMallocAsync((void**)&base, bytes, s));
    uint64_t* tsum = reinterpret_cast<uint64_t*>(base);
    uint64_t* s1 = tsum + n;
    uint64_t* N = s1 + n;
    unsigned long long* e5 = reinterpret_cast<unsigned long long*>(N + 11 * n);
    unsigned long long* e8 = e5 + m;
    unsigned long long* e9 = e8 + m;
    unsigned long long* e6a = e9 + m;
    int64_t* ebase = reinterpret_cast<int64_t*>(e6a + 2 * m);
    int32_t* up = reinterpret_cast<int32_t*>(ebase + n + 2);   // n + 2 int64 keep what follows 8-aligned
    int32_t* q_light = up + n;
    int32_t* q_heavy = q_light + n;
    // up, q_light and q_heavy hold 3n int32: round up to 8 bytes before the uint64 counters
    unsigned long long* qcnt = reinterpret_cast<unsigned long long*>(q_heavy + n + (n & 1));
    uint32_t* dense = reinterpret_cast<uint32_t*>(qcnt + 8);
    const OrbGraph G{ws.off, ws.cols, ws.deg, ws.offp, ws.colsp, ws.te};
    cudaError_t e = cudaMemsetAsync(base, 0, bytes, s);
    auto launched = [&]() {
        note_launch();
        if (e == cudaSuccess) e = cudaGetLastError();
    };
    if (e == cudaSuccess) {
        k_orb_tri<<<orb_grid(m), kOrbThreads, 0, s>>>(G, n, m, nullptr, nullptr, EdgeRoute{e5, e8, e9});
        launched();
    }
    if (e == cudaSuccess) {
        k_orb_vertex<<<orb_grid(n), kOrbThreads, 0, s>>>(G, n, tsum, s1, N);
        launched();
    }
    if (e == cudaSuccess) {
        k_orb_classify<<<orb_grid(n), kOrbThreads, 0, s>>>(G, n, q_light, q_heavy, qcnt);
        launched();
    }
    if (e == cudaSuccess) {
        k_orb_c4w<<<orb_grid(n), kOrbThreads, 0, s>>>(G, q_light, qcnt, nullptr, nullptr, e6a);
        launched();
    }
    if (e == cudaSuccess) {
        k_orb_c4b<<<heavy_blocks, kOrbThreads, 0, s>>>(G, n, q_heavy, qcnt, dense, nullptr, nullptr, e6a);
        launched();
    }
    if (e == cudaSuccess) {
        const int64_t blocks = (n + 255) / 256;
        k_eorb_up<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(g->off, g->cols, n, up);
        launched();
    }
    harp_status st = HARP_OK;
    if (e == cudaSuccess) st = exclusive_scan_i32_to_i64(up, ebase, n, ws.scan_tmp, ws.scan_tmp_len, s);
    if (e == cudaSuccess && st == HARP_OK) {
        const int64_t blocks = (m + 255) / 256;
        k_eorb_close<<<(unsigned)(blocks < (int64_t)num_sms() * 16 ? blocks : (int64_t)num_sms() * 16), 256, 0, s>>>(
            G, n, m, ws.dplus, tsum, s1, e5, e8, e9, e6a, ws.order, g->off, g->cols, up, ebase, d_out, ws.acc);
        launched();
    }
    cudaFreeAsync(base, s);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
    }
    return st;
}

}  // namespace harp
