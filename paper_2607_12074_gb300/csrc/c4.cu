// Step a5: the ordered-wedge anchor (Section III-B) and non-induced 4-cycles.
//
// In rank order, every 4-cycle has a unique top vertex u; its opposite corner x and both middle
// vertices w1, w2 rank below u.  For a root u, an ordered wedge is u - w - x with w in N-(u) and
// x in N(w), x < u; because rows are sorted in rank order, the x of one w are the prefix of w's row
// before u (length pos_w(u)).  With cnt(x) = number of wedges ending in x, the root contributes
// sum_x C(cnt(x), 2) 4-cycles.  Each increment adds the counter's previous value, which sums to the
// same total without a second pass.
//
// The frontier (the set of x) is not an induced class: whether u ~ x or w1 ~ w2 holds decides
// whether the cycle is induced, a diamond or part of a 4-clique; the closure resolves that mix
// (Section III-C explains why a frontier alone must not be reused as an induced state).
//
// Work per root W(u) = sum_{w in N-(u)} pos_w(u) decides the execution mode:
//   W <= warp_max           one warp, hash table in shared memory (warp-local mode)
//   W <= cta_max            one block, hash table in shared memory (CTA mode)
//   larger                  one block per (root, x-window): dense counters for a window of x in
//                           shared memory, 8/16/32-bit wide depending on d-(u) (cnt(x) <= d-(u))
#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int32_t kEmpty = -1;
constexpr int kWinThreads = 1024;
constexpr int kWinWords = 51200;             // 200 KiB of packed counters per window
constexpr int kMidThreads = 512;
constexpr int kMidSlots = 16384;             // 128 KiB hash table
constexpr int kSmallThreads = 256;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallSlots = 1024;            // per-warp hash table

__device__ __forceinline__ int counter_width(int64_t dminus) {
    return dminus <= 255 ? 8 : (dminus <= 65535 ? 16 : 32);
}

__device__ __forceinline__ int64_t window_span(int width) { return (int64_t)kWinWords * (32 / width); }

// Warp-cooperative traversal of 32 segments (lane l owns cols[base_l .. base_l + len_l)):
// flattened so that every lane takes one element per round.
template <typename F>
__device__ __forceinline__ void warp_flat(const int32_t* __restrict__ cols, int64_t base, int len, F&& f) {
    const int l = lane_id();
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (l >= o) incl += y;
    }
    const int excl = incl - len;
    const int total = __shfl_sync(kFull, incl, 31);
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + l;
        int o = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            const int e = __shfl_sync(kFull, excl, o + s);
            if (e <= t) o += s;
        }
        const int64_t ob = __shfl_sync(kFull, base, o);
        const int oe = __shfl_sync(kFull, excl, o);
        if (t < total) f(cols[ob + (t - oe)]);
    }
}

// shared-memory hash table: keys[] (kEmpty = free), cnt[]; returns the counter's previous value
__device__ __forceinline__ uint32_t hash_add(int32_t* keys, uint32_t* cnt, uint32_t mask, int32_t x) {
    uint32_t h = hash32((uint32_t)x) & mask;
    for (;;) {
        int32_t k = keys[h];
        if (k == kEmpty) {
            const int32_t prev = atomicCAS(&keys[h], kEmpty, x);
            if (prev == kEmpty || prev == x) return atomicAdd(&cnt[h], 1u);
            k = prev;
        }
        if (k == x) return atomicAdd(&cnt[h], 1u);
        h = (h + 1) & mask;
    }
}

// ---------------------------------------------------------------------------------------------
// Pass 1: every root (warp per root): W(u); small roots counted here, others queued.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSmallThreads) k_c4_small(const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ cols,
                                                            const int32_t* __restrict__ deg,
                                                            const int32_t* __restrict__ dplus, int64_t n,
                                                            uint32_t warp_max, uint32_t cta_max,
                                                            int32_t* __restrict__ q_mid,
                                                            int32_t* __restrict__ q_win,
                                                            int32_t* __restrict__ wcount,
                                                            uint64_t* __restrict__ acc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* my_keys = reinterpret_cast<int32_t*>(smem_raw) + (threadIdx.x >> 5) * kSmallSlots;
    uint32_t* my_cnt = reinterpret_cast<uint32_t*>(smem_raw + kSmallWarps * kSmallSlots * sizeof(int32_t)) +
                       (threadIdx.x >> 5) * kSmallSlots;
    __shared__ uint64_t red[32];
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t wid = (int64_t)blockIdx.x * kSmallWarps + w;
    const int64_t nw = (int64_t)gridDim.x * kSmallWarps;
    unsigned long long* qcnt_mid = (unsigned long long*)&acc[Q_C4_MID];
    unsigned long long* qcnt_win = (unsigned long long*)&acc[Q_C4_WIN];
    uint64_t c4 = 0;
    for (int64_t k = wid; k < n; k += nw) {
        const int32_t u = (int32_t)(n - 1 - k);  // descending rank: heavy roots queued first
        const int64_t dm = (int64_t)deg[u] - dplus[u];
        if (dm < 2) continue;
        const int64_t ub = off[u];
        // W(u) = sum over w in N-(u) of pos_w(u)
        uint64_t W = 0;
        for (int64_t a = l; a < dm; a += 32) {
            const int32_t wv = cols[ub + a];
            const int64_t wb = off[wv];
            W += (uint64_t)lower_bound_i32(cols + wb, off[wv + 1] - wb, u);
        }
        W = warp_sum(W);
        if (W == 0) continue;
        if (W > warp_max) {
            if (l == 0) {
                if (W <= cta_max) {
                    const unsigned long long slot = atomicAdd(qcnt_mid, 1ull);
                    q_mid[slot] = u;
                    q_mid[n + slot] = (int32_t)W;  // second half: work, sizes the CTA table
                } else {
                    const unsigned long long slot = atomicAdd(qcnt_win, 1ull);
                    q_win[slot] = u;
                    const int64_t span = window_span(counter_width(dm));
                    wcount[slot] = (int32_t)(((int64_t)u + span - 1) / span);
                }
            }
            continue;
        }
        uint32_t P = 32;
        while (P < 2 * W) P <<= 1;
        for (uint32_t i = l; i < P; i += 32) {
            my_keys[i] = kEmpty;
            my_cnt[i] = 0;
        }
        __syncwarp();
        for (int64_t a0 = 0; a0 < dm; a0 += 32) {
            const int64_t a = a0 + l;
            int64_t base = 0;
            int len = 0;
            if (a < dm) {
                const int32_t wv = cols[ub + a];
                base = off[wv];
                len = (int)lower_bound_i32(cols + base, off[wv + 1] - base, u);
            }
            warp_flat(cols, base, len, [&](int32_t x) { c4 += hash_add(my_keys, my_cnt, P - 1, x); });
        }
        __syncwarp();
    }
    c4 = block_sum_u64(c4, red);
    if (threadIdx.x == 0 && c4) atomicAdd((unsigned long long*)&acc[ACC_C4], (unsigned long long)c4);
}

// ---------------------------------------------------------------------------------------------
// CTA mode: one block per queued root, shared-memory hash table.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kMidThreads) k_c4_mid(const int64_t* __restrict__ off,
                                                        const int32_t* __restrict__ cols,
                                                        const int32_t* __restrict__ deg,
                                                        const int32_t* __restrict__ dplus,
                                                        const int32_t* __restrict__ q_mid, int64_t n,
                                                        uint64_t* __restrict__ acc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem_raw + kMidSlots * sizeof(int32_t));
    __shared__ int64_t s_item;
    __shared__ uint64_t red[32];
    const int w = threadIdx.x >> 5;
    constexpr int NW = kMidThreads / 32;
    const int64_t nq = (int64_t)acc[Q_C4_MID];
    unsigned long long* ticket = (unsigned long long*)&acc[T_C4_MID];
    uint64_t c4 = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(ticket, 1ull);
        __syncthreads();
        const int64_t k = s_item;
        __syncthreads();
        if (k >= nq) break;
        const int32_t u = q_mid[k];
        const int64_t dm = (int64_t)deg[u] - dplus[u];
        const int64_t ub = off[u];
        // table size: next power of two >= 2 W (distinct x <= W), at most kMidSlots
        const uint32_t W = (uint32_t)q_mid[n + k];
        uint32_t P = 64;
        while (P < 2 * W && P < (uint32_t)kMidSlots) P <<= 1;
        for (uint32_t i = threadIdx.x; i < P; i += kMidThreads) {
            keys[i] = kEmpty;
            cnt[i] = 0;
        }
        __syncthreads();
        for (int64_t a0 = (int64_t)w * 32; a0 < dm; a0 += (int64_t)NW * 32) {
            const int64_t a = a0 + lane_id();
            int64_t base = 0;
            int len = 0;
            if (a < dm) {
                const int32_t wv = cols[ub + a];
                base = off[wv];
                len = (int)lower_bound_i32(cols + base, off[wv + 1] - base, u);
            }
            warp_flat(cols, base, len, [&](int32_t x) { c4 += hash_add(keys, cnt, P - 1, x); });
        }
        __syncthreads();
    }
    c4 = block_sum_u64(c4, red);
    if (threadIdx.x == 0 && c4) atomicAdd((unsigned long long*)&acc[ACC_C4], (unsigned long long)c4);
}

// ---------------------------------------------------------------------------------------------
// Windowed CTA mode: one block per (root, window of x); dense packed counters in shared memory.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kWinThreads) k_c4_window(const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ cols,
                                                           const int32_t* __restrict__ deg,
                                                           const int32_t* __restrict__ dplus,
                                                           const int32_t* __restrict__ q_win,
                                                           const int64_t* __restrict__ win_prefix,
                                                           uint64_t* __restrict__ acc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* cw = reinterpret_cast<uint32_t*>(smem_raw);
    __shared__ int64_t s_item;
    __shared__ uint64_t red[32];
    const int w = threadIdx.x >> 5;
    constexpr int NW = kWinThreads / 32;
    const int64_t nroots = (int64_t)acc[Q_C4_WIN];
    const int64_t total = win_prefix[nroots];
    unsigned long long* ticket = (unsigned long long*)&acc[T_C4_WIN];
    uint64_t c4 = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(ticket, 1ull);
        __syncthreads();
        const int64_t t = s_item;
        __syncthreads();
        if (t >= total) break;
        // root index: last k with win_prefix[k] <= t
        int64_t lo = 0, hi = nroots;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (win_prefix[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int32_t u = q_win[lo];
        const int64_t win = t - win_prefix[lo];
        const int64_t dm = (int64_t)deg[u] - dplus[u];
        const int width = counter_width(dm);
        const int64_t span = window_span(width);
        const int32_t xlo = (int32_t)(win * span);
        const int64_t xhi64 = (win + 1) * span < (int64_t)u ? (win + 1) * span : (int64_t)u;
        const int32_t xhi = (int32_t)xhi64;
        const int words = (int)((xhi64 - xlo + (32 / width) - 1) / (32 / width));
        for (int i = threadIdx.x; i < words; i += kWinThreads) cw[i] = 0;
        __syncthreads();
        const int64_t ub = off[u];
        for (int64_t a0 = (int64_t)w * 32; a0 < dm; a0 += (int64_t)NW * 32) {
            const int64_t a = a0 + lane_id();
            int64_t base = 0;
            int len = 0;
            if (a < dm) {
                const int32_t wv = cols[ub + a];
                const int64_t wb = off[wv];
                const int64_t wl = off[wv + 1] - wb;
                const int64_t p0 = lower_bound_i32(cols + wb, wl, xlo);
                const int64_t p1 = lower_bound_i32(cols + wb, wl, xhi);
                base = wb + p0;
                len = (int)(p1 - p0);
            }
            if (width == 8) {
                warp_flat(cols, base, len, [&](int32_t x) {
                    const uint32_t r = (uint32_t)(x - xlo), sh = (r & 3u) * 8u;
                    c4 += (atomicAdd(&cw[r >> 2], 1u << sh) >> sh) & 0xffu;
                });
            } else if (width == 16) {
                warp_flat(cols, base, len, [&](int32_t x) {
                    const uint32_t r = (uint32_t)(x - xlo), sh = (r & 1u) * 16u;
                    c4 += (atomicAdd(&cw[r >> 1], 1u << sh) >> sh) & 0xffffu;
                });
            } else {
                warp_flat(cols, base, len, [&](int32_t x) { c4 += atomicAdd(&cw[x - xlo], 1u); });
            }
        }
        __syncthreads();
    }
    c4 = block_sum_u64(c4, red);
    if (threadIdx.x == 0 && c4) atomicAdd((unsigned long long*)&acc[ACC_C4], (unsigned long long)c4);
}

}  // namespace

harp_status count_wedge_c4(const harp_csr* g, Workspace& ws, const harp_plan& plan, cudaStream_t s) {
    const int64_t n = g->n;
    if (n == 0 || g->m == 0) return HARP_OK;
    uint32_t warp_max = plan.c4_warp_max_work ? plan.c4_warp_max_work : 512;
    if (warp_max > kSmallSlots / 2) warp_max = kSmallSlots / 2;
    uint32_t cta_max = plan.c4_cta_max_work ? plan.c4_cta_max_work : kMidSlots / 2;
    if (cta_max > kMidSlots / 2) cta_max = kMidSlots / 2;
    if (cta_max < warp_max) cta_max = warp_max;

    HARP_CK(cudaMemsetAsync(ws.q_win + n, 0, (size_t)n * sizeof(int32_t), s));  // wcount
    int32_t* wcount = ws.q_win + n;
    const size_t small_smem = (size_t)kSmallWarps * kSmallSlots * (sizeof(int32_t) + sizeof(uint32_t));
    HARP_CK(cudaFuncSetAttribute(k_c4_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem));
    k_c4_small<<<152 * 3, kSmallThreads, small_smem, s>>>(ws.off, ws.cols, ws.deg, ws.dplus, n, warp_max,
                                                          cta_max, ws.q_mid, ws.q_win, wcount, ws.acc);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_SMALL));
    const size_t mid_smem = (size_t)kMidSlots * (sizeof(int32_t) + sizeof(uint32_t));
    HARP_CK(cudaFuncSetAttribute(k_c4_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mid_smem));
    k_c4_mid<<<152, kMidThreads, mid_smem, s>>>(ws.off, ws.cols, ws.deg, ws.dplus, ws.q_mid, n, ws.acc);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_MID));
    HARP_TRY(exclusive_scan_i32_to_i64(wcount, ws.win_prefix, n, ws.scan_tmp, ws.scan_tmp_len, s));
    const size_t win_smem = (size_t)kWinWords * sizeof(uint32_t);
    HARP_CK(cudaFuncSetAttribute(k_c4_window, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem));
    k_c4_window<<<152, kWinThreads, win_smem, s>>>(ws.off, ws.cols, ws.deg, ws.dplus, ws.q_win, ws.win_prefix,
                                                   ws.acc);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_WINDOW));
    return HARP_OK;
}

}  // namespace harp
