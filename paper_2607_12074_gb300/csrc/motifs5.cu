// Connected induced 5-vertex motif counts (the paper's future work, Section VI), by explicit
// enumeration of every connected 5-vertex subset once on the GPU.
//
// An induced occurrence is a 5-vertex subset S with G[S] connected (Section II).  A labelled graph on
// five vertices is a 10-bit mask, bit k for the k-th vertex pair (i, j), i < j, in lexicographic
// order; its class key is the smallest mask over the 120 vertex permutations, and the 21 connected
// classes are numbered in increasing (edge count, key) order.  The host builds the 1024-entry table
// mask -> class (255 for a disconnected mask) from that definition once, and passes it to the kernel.
//
// Enumeration: Wernicke's ESU (2006) in rank order (after the shared orientation pass, ids are ranks).
// A subset is enumerated from its lowest-ranked vertex v (the root): extensions only take vertices
// above v, and a vertex w added to the subset S contributes its exclusive neighbours, those of N(w)
// above v outside N[S]; each connected 5-subset is produced exactly once.  One warp per root: the
// root's first-level children (one per out-neighbour w1 of v, carrying the out-neighbours before w1)
// are dealt to the lanes, and each lane walks the three remaining levels with its extension sets in
// its own slice of a global scratch (bounded by the maximum degree: |E_2| <= 2D, |E_3| <= 3D,
// |E_4| <= 4D).  At five vertices the lane reads the ten adjacencies of S by binary search, looks the
// mask up and counts the class in the warp's shared histogram.
//
// The work is the number of connected 5-subsets (times about ten binary searches), which explodes on
// graphs with hubs: this path is for small and sparse graphs.  The closure-derived alternative the
// paper names (a 5-vertex analogue of Section III-F) is not built.
#include <algorithm>
#include <mutex>
#include <vector>

#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kM5Classes = 21;
constexpr int kM5Threads = 256;
constexpr int kM5Warps = kM5Threads / 32;

struct M5Table {
    uint8_t cls[1024];  // mask -> class index, 255 = disconnected
};

// the table and the classes' keys, built once on the host from the definition above
struct M5Host {
    M5Table table;
    uint16_t keys[kM5Classes];
};

const M5Host& m5_host() {
    static M5Host h;
    static std::once_flag once;
    std::call_once(once, [] {
        int pi[10], pj[10], bit[5][5];
        for (int i = 0, k = 0; i < 5; ++i)
            for (int j = i + 1; j < 5; ++j, ++k) {
                pi[k] = i;
                pj[k] = j;
                bit[i][j] = bit[j][i] = k;
            }
        std::vector<int> canon(1024, -1);
        int perm[5] = {0, 1, 2, 3, 4};
        std::vector<std::vector<int>> perms;
        do perms.emplace_back(perm, perm + 5);
        while (std::next_permutation(perm, perm + 5));
        for (int mask = 0; mask < 1024; ++mask) {
            // connected?
            int seen = 1, grow = 1;
            while (grow) {
                grow = 0;
                for (int k = 0; k < 10; ++k)
                    if ((mask >> k) & 1) {
                        const int a = 1 << pi[k], b = 1 << pj[k];
                        if (((seen & a) != 0) != ((seen & b) != 0)) {
                            seen |= a | b;
                            grow = 1;
                        }
                    }
            }
            if (seen != 31) continue;
            int best = 1024;
            for (const auto& p : perms) {
                int m2 = 0;
                for (int k = 0; k < 10; ++k)
                    if ((mask >> k) & 1) m2 |= 1 << bit[p[pi[k]]][p[pj[k]]];
                best = std::min(best, m2);
            }
            canon[mask] = best;
        }
        std::vector<int> keys;
        for (int mask = 0; mask < 1024; ++mask)
            if (canon[mask] == mask) keys.push_back(mask);
        std::sort(keys.begin(), keys.end(), [](int a, int b) {
            const int ca = __builtin_popcount(a), cb = __builtin_popcount(b);
            return ca != cb ? ca < cb : a < b;
        });
        for (int mask = 0; mask < 1024; ++mask) {
            h.table.cls[mask] = 255;
            if (canon[mask] < 0) continue;
            const int c = (int)(std::find(keys.begin(), keys.end(), canon[mask]) - keys.begin());
            h.table.cls[mask] = (uint8_t)c;
        }
        for (int c = 0; c < (int)keys.size() && c < kM5Classes; ++c) h.keys[c] = (uint16_t)keys[c];
    });
    return h;
}

__device__ __forceinline__ bool adj(const int64_t* __restrict__ off, const int32_t* __restrict__ cols, int32_t a,
                                    int32_t b) {
    const int64_t rb = off[a], re = off[a + 1];
    const int64_t p = rb + lower_bound_i32(cols + rb, re - rb, b);
    return p < re && __ldg(cols + p) == b;
}

// v is not in S[0..s) and adjacent to none of them
__device__ __forceinline__ bool outside_closed(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                               const int32_t* S, int s, int32_t y) {
    for (int i = 0; i < s; ++i)
        if (y == S[i] || adj(off, cols, S[i], y)) return false;
    return true;
}

// E_next = E[0 .. keep) followed by the exclusive neighbours of w (above root, outside N[S[0..s)]);
// E and E_next are strided slices (element j at [j * stride]); returns |E_next|
__device__ __forceinline__ int extend(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                      const int32_t* E, int keep, int32_t* En, int64_t stride, const int32_t* S,
                                      int s, int32_t w, int32_t root) {
    for (int j = 0; j < keep; ++j) En[j * stride] = E[j * stride];
    int len = keep;
    const int64_t wb = off[w], we = off[w + 1];
    for (int64_t p = wb + lower_bound_i32(cols + wb, we - wb, root + 1); p < we; ++p) {
        const int32_t y = __ldg(cols + p);
        if (outside_closed(off, cols, S, s, y)) En[(len++) * stride] = y;
    }
    return len;
}

__global__ void __launch_bounds__(kM5Threads) k_m5_esu(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                                       int64_t n, M5Table table, int32_t* __restrict__ scratch,
                                                       int64_t D, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long hist[kM5Warps][kM5Classes];
    __shared__ uint8_t cls[1024];
    for (int i = threadIdx.x; i < 1024; i += kM5Threads) cls[i] = table.cls[i];
    for (int i = threadIdx.x; i < kM5Warps * kM5Classes; i += kM5Threads) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t T = (int64_t)gridDim.x * blockDim.x;                   // threads = scratch stride
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t* E2 = scratch + tid;                                         // 2D entries
    int32_t* E3 = E2 + 2 * D * T;                                        // 3D entries
    int32_t* E4 = E3 + 3 * D * T;                                        // 4D entries
    const int64_t nw = T >> 5;
    for (int64_t v = tid >> 5; v < n; v += nw) {
        const int64_t vb = off[v], ve = off[v + 1];
        const int64_t first_up = vb + lower_bound_i32(cols + vb, ve - vb, (int32_t)v + 1);
        const int L = (int)(ve - first_up);  // out-neighbours of v: the first-level extension set
        for (int i1 = l; i1 < L; i1 += 32) {
            int32_t S[5];
            S[0] = (int32_t)v;
            S[1] = __ldg(cols + first_up + i1);
            // E2 = out-neighbours before w1, then w1's exclusive neighbours relative to N[{v}]
            int n2 = 0;
            for (int j = 0; j < i1; ++j) E2[(n2++) * T] = __ldg(cols + first_up + j);
            {
                const int64_t wb = off[S[1]], we = off[S[1] + 1];
                for (int64_t p = wb + lower_bound_i32(cols + wb, we - wb, (int32_t)v + 1); p < we; ++p) {
                    const int32_t y = __ldg(cols + p);
                    if (outside_closed(off, cols, S, 1, y)) E2[(n2++) * T] = y;
                }
            }
            for (int i2 = n2 - 1; i2 >= 0; --i2) {
                S[2] = E2[i2 * T];
                const int n3 = extend(off, cols, E2, i2, E3, T, S, 2, S[2], (int32_t)v);
                for (int i3 = n3 - 1; i3 >= 0; --i3) {
                    S[3] = E3[i3 * T];
                    const int n4 = extend(off, cols, E3, i3, E4, T, S, 3, S[3], (int32_t)v);
                    for (int i4 = n4 - 1; i4 >= 0; --i4) {
                        S[4] = E4[i4 * T];
                        int mask = 0;
#pragma unroll
                        for (int a = 0, k = 0; a < 5; ++a)
#pragma unroll
                            for (int b = a + 1; b < 5; ++b, ++k)
                                if (adj(off, cols, S[a], S[b])) mask |= 1 << k;
                        const int c = cls[mask];
                        if (c < kM5Classes) atomicAdd(&hist[w][c], 1ull);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kM5Classes; c += kM5Threads) {
        unsigned long long t = 0;
        for (int k = 0; k < kM5Warps; ++k) t += hist[k][c];
        if (t) atomicAdd(&out[c], t);
    }
}

}  // namespace
}  // namespace harp

using namespace harp;

extern "C" harp_status harp_motif5_classes(uint16_t keys_out[21]) {
    if (!keys_out) return HARP_EINVAL;
    const M5Host& h = m5_host();
    for (int c = 0; c < kM5Classes; ++c) keys_out[c] = h.keys[c];
    return HARP_OK;
}

extern "C" harp_status harp_count5(const harp_csr* gc, uint64_t counts_out[21]) {
    if (!gc || !counts_out) return HARP_EINVAL;
    harp_csr* g = const_cast<harp_csr*>(gc);
    if (g->n < 5 || g->m < 4) {
        for (int c = 0; c < kM5Classes; ++c) counts_out[c] = 0;
        return HARP_OK;
    }
    HARP_CK(cudaSetDevice(g->device));
    cudaStream_t s = g->stream;
    const M5Host& h = m5_host();
    HARP_TRY(ws_ensure(g->ws, g->n, g->m, s));
    Workspace& ws = g->ws;
    HARP_CK(cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s));
    HARP_TRY(orient(g, ws, s));  // ranks: ESU roots are the lowest-ranked vertex of each subset
    // per-thread extension sets: 9 D int32 a thread, at most 4 GiB in all
    const int64_t D = g->max_deg > 0 ? g->max_deg : 1;
    int64_t blocks = (int64_t)num_sms() * 4;
    while (blocks > 1 && (size_t)blocks * kM5Threads * 9 * (size_t)D * 4 > ((size_t)4 << 30)) blocks >>= 1;
    const int64_t warps_needed = (g->n + 0) / 1;  // one warp per root
    if (blocks * kM5Warps > warps_needed) blocks = (warps_needed + kM5Warps - 1) / kM5Warps;
    if (blocks < 1) blocks = 1;
    const size_t scratch_bytes = (size_t)blocks * kM5Threads * 9 * (size_t)D * sizeof(int32_t);
    int32_t* scratch = nullptr;
    unsigned long long* d_out = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, scratch_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_out, sizeof(unsigned long long) * kM5Classes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, sizeof(unsigned long long) * kM5Classes, s);
    if (e == cudaSuccess) {
        k_m5_esu<<<(unsigned)blocks, kM5Threads, 0, s>>>(ws.off, ws.cols, g->n, h.table, scratch, D, d_out);
        note_launch();
        e = cudaGetLastError();
    }
    uint64_t host[kM5Classes];
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, d_out, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (scratch) cudaFreeAsync(scratch, s);
    if (d_out) cudaFreeAsync(d_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
    }
    for (int c = 0; c < kM5Classes; ++c) counts_out[c] = host[c];
    return HARP_OK;
}
