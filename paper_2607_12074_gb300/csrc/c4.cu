// Step a5: the ordered-wedge anchor (Section III-B) and non-induced 4-cycles.
//
// In rank order, every 4-cycle has a unique top vertex u; its opposite corner x and both middle
// vertices w1, w2 rank below u.  For a root u, an ordered wedge is u - w - x with w in N-(u) and
// x in N(w), x < u; because rows are sorted in rank order, the x of one w are a contiguous range of
// w's row ending at pos_w(u), the position of u in that row.  With cnt(x) = number of wedges ending
// in x, the root contributes sum_x C(cnt(x), 2) 4-cycles; each increment adds the counter's previous
// value, which sums to the same total without a second pass.
//
// Two bounds shape the work: cnt(x) <= d(x) (every wedge into x uses a distinct neighbour of x) and
// cnt(x) <= d-(u).  Hence
//   * x of degree 1 never complete a cycle: the x-range is [n1, u) with n1 the first rank of
//     degree >= 2 (rank order puts isolated vertices and leaves first), and every row's segment
//     starts at fpos[w] (the first neighbour of degree >= 2, found once when the row was sorted);
//   * a dense counter for x fits 8 bits if d(x) <= 255 or d-(u) <= 255, 16 bits below 65536.  Rank
//     order makes degree monotone in x, so the x-range splits into at most three bands
//     [n1, r256), [r256, r64k), [r64k, u) whose counters are 8, 16 and 32 bits wide (narrower when
//     d-(u) allows), and most of rank space is covered by 8-bit windows.
//
// The frontier (the set of x) is not an induced class: whether u ~ x or w1 ~ w2 holds decides
// whether the cycle is induced, a diamond or part of a 4-clique; the closure resolves that mix
// (Section III-C explains why a frontier alone must not be reused as an induced state).
//
// Work per root W(u) = sum_{w in N-(u)} (pos_w(u) - fpos[w]) decides the execution mode:
//   W <= warp_max           one warp, hash table in shared memory (warp-local mode)
//   W <= cta_max            one block, hash table in shared memory (CTA mode)
//   larger                  one block per (root, x-window): dense packed counters in shared memory
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
constexpr int kLong = 32;                    // segments at least this long are read warp-coalesced

// first rank whose degree is > t (deg is non-decreasing in rank order)
__device__ __forceinline__ int64_t rank_above(const int32_t* __restrict__ deg, int64_t n, int32_t t) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (deg[mid] <= t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct Bands {
    int64_t n1, r256, r64k;  // first rank of degree >= 2, >= 256, >= 65536
};

__device__ __forceinline__ Bands load_bands(const int32_t* __restrict__ deg, int64_t n) {
    Bands b;
    b.n1 = rank_above(deg, n, 1);
    b.r256 = rank_above(deg, n, 255);
    b.r64k = rank_above(deg, n, 65535);
    return b;
}

__device__ __forceinline__ int width_for(int band, int64_t dm) {
    const int by_dm = dm <= 255 ? 8 : (dm <= 65535 ? 16 : 32);
    const int by_x = band == 0 ? 8 : (band == 1 ? 16 : 32);
    return by_dm < by_x ? by_dm : by_x;
}

__device__ __forceinline__ int64_t span_for(int width) { return (int64_t)kWinWords * (32 / width); }

// The x-range [n1, u) of root u as bands; returns band b's [lo, hi) (empty if lo >= hi).
__device__ __forceinline__ void band_range(const Bands& B, int band, int64_t u, int64_t& lo, int64_t& hi) {
    const int64_t a[4] = {B.n1, B.r256 > B.n1 ? B.r256 : B.n1, B.r64k > B.n1 ? B.r64k : B.n1, u};
    lo = a[band] < u ? a[band] : u;
    hi = a[band + 1] < u ? a[band + 1] : u;
    if (band == 2) hi = u;
    if (hi < lo) hi = lo;
}

__device__ __forceinline__ int64_t window_count(const Bands& B, int64_t u, int64_t dm) {
    int64_t total = 0;
    for (int band = 0; band < 3; ++band) {
        int64_t lo, hi;
        band_range(B, band, u, lo, hi);
        if (hi > lo) {
            const int64_t span = span_for(width_for(band, dm));
            total += (hi - lo + span - 1) / span;
        }
    }
    return total;
}

// position of u in w's row, for w < u: u lies in the out-list N+(w)
__device__ __forceinline__ int64_t pos_of_root(const int64_t* __restrict__ offp, const int32_t* __restrict__ colsp,
                                               const int32_t* __restrict__ deg, const int32_t* __restrict__ dplus,
                                               int32_t w, int32_t u) {
    const int64_t pb = offp[w];
    return (int64_t)(deg[w] - dplus[w]) + lower_bound_i32(colsp + pb, offp[w + 1] - pb, u);
}

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
        if (t < total) f(__ldg(cols + ob + (t - oe)));
    }
}

// Long segments one after the other, each read by the whole warp (coalesced); short ones flattened.
template <typename F>
__device__ __forceinline__ void warp_segments(const int32_t* __restrict__ cols, int64_t base, int len, F&& f) {
    const int l = lane_id();
    uint32_t longs = __ballot_sync(kFull, len >= kLong);
    while (longs) {
        const int src = __ffs(longs) - 1;
        longs &= longs - 1;
        const int64_t b = __shfl_sync(kFull, base, src);
        const int n = __shfl_sync(kFull, len, src);
        for (int k = l; k < n; k += 32) f(__ldg(cols + b + k));
    }
    warp_flat(cols, base, len >= kLong ? 0 : len, f);
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
                                                            const int64_t* __restrict__ offp,
                                                            const int32_t* __restrict__ colsp,
                                                            const int32_t* __restrict__ deg,
                                                            const int32_t* __restrict__ dplus,
                                                            const int32_t* __restrict__ fpos, int64_t n,
                                                            uint32_t warp_max, uint32_t cta_max,
                                                            int32_t* __restrict__ q_mid,
                                                            int32_t* __restrict__ q_win,
                                                            int32_t* __restrict__ wcount,
                                                            uint64_t* __restrict__ acc, Sink sink) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* my_keys = reinterpret_cast<int32_t*>(smem_raw) + (threadIdx.x >> 5) * kSmallSlots;
    uint32_t* my_cnt = reinterpret_cast<uint32_t*>(smem_raw + kSmallWarps * kSmallSlots * sizeof(int32_t)) +
                       (threadIdx.x >> 5) * kSmallSlots;
    __shared__ uint64_t red[32];
    __shared__ Bands sB;
    if (threadIdx.x == 0) sB = load_bands(deg, n);
    __syncthreads();
    const Bands B = sB;
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t wid = (int64_t)blockIdx.x * kSmallWarps + w;
    const int64_t nw = (int64_t)gridDim.x * kSmallWarps;
    unsigned long long* qcnt_mid = (unsigned long long*)&acc[Q_C4_MID];
    unsigned long long* qcnt_win = (unsigned long long*)&acc[Q_C4_WIN];
    uint64_t c4 = 0;
    for (int64_t k = wid; k < n - B.n1; k += nw) {
        const int32_t u = (int32_t)(n - 1 - k);  // descending rank: heavy roots queued first
        const int64_t dm = (int64_t)deg[u] - dplus[u];
        if (dm < 2) continue;
        const int64_t ub = off[u];
        // W(u) = sum over w in N-(u) of the segment lengths pos_w(u) - fpos[w]
        uint64_t W = 0;
        for (int64_t a = l; a < dm; a += 32) {
            const int32_t wv = cols[ub + a];
            const int64_t p = pos_of_root(offp, colsp, deg, dplus, wv, u);
            const int64_t f = fpos[wv];
            W += p > f ? (uint64_t)(p - f) : 0;
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
                    wcount[slot] = (int32_t)window_count(B, u, dm);
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
        uint64_t a_c4 = 0;
        for (int64_t a0 = 0; a0 < dm; a0 += 32) {
            const int64_t a = a0 + l;
            int64_t base = 0;
            int len = 0;
            if (a < dm) {
                const int32_t wv = cols[ub + a];
                const int64_t p = pos_of_root(offp, colsp, deg, dplus, wv, u);
                const int64_t f = fpos[wv];
                base = off[wv] + f;
                len = p > f ? (int)(p - f) : 0;
            }
            warp_flat(cols, base, len, [&](int32_t x) { a_c4 += hash_add(my_keys, my_cnt, P - 1, x); });
        }
        if (sink.batch()) {
            a_c4 = warp_sum(a_c4);
            if (l == 0) sink_add(sink, u, G_C4, a_c4);
        } else {
            c4 += a_c4;
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
                                                        const int64_t* __restrict__ offp,
                                                        const int32_t* __restrict__ colsp,
                                                        const int32_t* __restrict__ deg,
                                                        const int32_t* __restrict__ dplus,
                                                        const int32_t* __restrict__ fpos,
                                                        const int32_t* __restrict__ q_mid, int64_t n,
                                                        uint64_t* __restrict__ acc, Sink sink) {
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
        uint64_t a_c4 = 0;
        for (int64_t a0 = (int64_t)w * 32; a0 < dm; a0 += (int64_t)NW * 32) {
            const int64_t a = a0 + lane_id();
            int64_t base = 0;
            int len = 0;
            if (a < dm) {
                const int32_t wv = cols[ub + a];
                const int64_t p = pos_of_root(offp, colsp, deg, dplus, wv, u);
                const int64_t f = fpos[wv];
                base = off[wv] + f;
                len = p > f ? (int)(p - f) : 0;
            }
            warp_segments(cols, base, len, [&](int32_t x) { a_c4 += hash_add(keys, cnt, P - 1, x); });
        }
        __syncthreads();
        if (sink.batch()) {
            const uint64_t t = block_sum_u64(a_c4, red);
            if (threadIdx.x == 0) sink_add(sink, u, G_C4, t);
        } else {
            c4 += a_c4;
        }
    }
    c4 = block_sum_u64(c4, red);
    if (threadIdx.x == 0 && c4) atomicAdd((unsigned long long*)&acc[ACC_C4], (unsigned long long)c4);
}

// ---------------------------------------------------------------------------------------------
// Windowed CTA mode: one block per (root, window of x); dense packed counters in shared memory.
// Groups of 32 lower neighbours are handed to warps dynamically, heaviest (highest-degree) first.
// ---------------------------------------------------------------------------------------------
template <int WIDTH>
__device__ __forceinline__ uint32_t counter_add(uint32_t* cw, uint32_t r) {
    if (WIDTH == 8) {
        const uint32_t sh = (r & 3u) << 3;
        return (atomicAdd(&cw[r >> 2], 1u << sh) >> sh) & 0xffu;
    } else if (WIDTH == 16) {
        const uint32_t sh = (r & 1u) << 4;
        return (atomicAdd(&cw[r >> 1], 1u << sh) >> sh) & 0xffffu;
    } else {
        return atomicAdd(&cw[r], 1u);
    }
}

template <int WIDTH>
__device__ __forceinline__ void window_pass(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                            const int64_t* __restrict__ offp, const int32_t* __restrict__ colsp,
                                            const int32_t* __restrict__ deg, const int32_t* __restrict__ dplus,
                                            const int32_t* __restrict__ fpos, int32_t u, int64_t ub, int64_t dm,
                                            int32_t xlo, int32_t xhi, bool first, bool last, uint32_t* cw,
                                            int* s_group, uint64_t& c4) {
    const int l = lane_id();
    const int ngroups = (int)((dm + 31) >> 5);
    for (;;) {
        int g = 0;
        if (l == 0) g = atomicAdd(s_group, 1);
        g = __shfl_sync(kFull, g, 0);
        if (g >= ngroups) break;
        const int64_t a = (int64_t)(ngroups - 1 - g) * 32 + l;  // heaviest groups first
        int64_t base = 0;
        int len = 0;
        if (a < dm) {
            const int32_t wv = cols[ub + a];
            const int64_t wb = off[wv];
            const int64_t rowlen = off[wv + 1] - wb;
            const int64_t p0 = first ? (int64_t)fpos[wv] : lower_bound_i32(cols + wb, rowlen, xlo);
            const int64_t p1 = last ? pos_of_root(offp, colsp, deg, dplus, wv, u)
                                    : lower_bound_i32(cols + wb, rowlen, xhi);
            base = wb + p0;
            len = p1 > p0 ? (int)(p1 - p0) : 0;
        }
        warp_segments(cols, base, len, [&](int32_t x) { c4 += counter_add<WIDTH>(cw, (uint32_t)(x - xlo)); });
    }
}

__global__ void __launch_bounds__(kWinThreads, 1) k_c4_window(const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ cols,
                                                           const int64_t* __restrict__ offp,
                                                           const int32_t* __restrict__ colsp,
                                                           const int32_t* __restrict__ deg,
                                                           const int32_t* __restrict__ dplus,
                                                           const int32_t* __restrict__ fpos, int64_t n,
                                                           const int32_t* __restrict__ q_win,
                                                           const int64_t* __restrict__ win_prefix,
                                                           uint64_t* __restrict__ acc, Sink sink) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* cw = reinterpret_cast<uint32_t*>(smem_raw);
    __shared__ int64_t s_item;
    __shared__ int s_group;
    __shared__ uint64_t red[32];
    __shared__ Bands sB;
    if (threadIdx.x == 0) sB = load_bands(deg, n);
    __syncthreads();
    const Bands B = sB;
    const int64_t nroots = (int64_t)acc[Q_C4_WIN];
    const int64_t total = win_prefix[nroots];
    unsigned long long* ticket = (unsigned long long*)&acc[T_C4_WIN];
    uint64_t c4 = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = (int64_t)atomicAdd(ticket, 1ull);
            s_group = 0;
        }
        __syncthreads();
        const int64_t t = s_item;
        if (t >= total) break;
        // root index: last k with win_prefix[k] <= t
        int64_t lo = 0, hi = nroots;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (win_prefix[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int32_t u = q_win[lo];
        const int64_t dm = (int64_t)deg[u] - dplus[u];
        // window j of the root, located in its bands
        int64_t j = t - win_prefix[lo];
        int width = 32;
        int64_t xlo = 0, xhi = 0;
        for (int band = 0; band < 3; ++band) {
            int64_t blo, bhi;
            band_range(B, band, u, blo, bhi);
            if (bhi <= blo) continue;
            const int wd = width_for(band, dm);
            const int64_t span = span_for(wd);
            const int64_t nb = (bhi - blo + span - 1) / span;
            if (j < nb) {
                width = wd;
                xlo = blo + j * span;
                xhi = xlo + span < bhi ? xlo + span : bhi;
                break;
            }
            j -= nb;
        }
        const int per = 32 / width;
        const int words = (int)((xhi - xlo + per - 1) / per);
        for (int i = threadIdx.x; i < words; i += kWinThreads) cw[i] = 0;
        __syncthreads();
        const int64_t ub = off[u];
        const bool first = xlo == B.n1;
        const bool last = xhi == (int64_t)u;
        uint64_t a_c4 = 0;
        if (width == 8)
            window_pass<8>(off, cols, offp, colsp, deg, dplus, fpos, u, ub, dm, (int32_t)xlo, (int32_t)xhi, first,
                           last, cw, &s_group, a_c4);
        else if (width == 16)
            window_pass<16>(off, cols, offp, colsp, deg, dplus, fpos, u, ub, dm, (int32_t)xlo, (int32_t)xhi, first,
                            last, cw, &s_group, a_c4);
        else
            window_pass<32>(off, cols, offp, colsp, deg, dplus, fpos, u, ub, dm, (int32_t)xlo, (int32_t)xhi, first,
                            last, cw, &s_group, a_c4);
        __syncthreads();
        if (sink.batch()) {
            const uint64_t t = block_sum_u64(a_c4, red);
            if (threadIdx.x == 0) sink_add(sink, u, G_C4, t);
        } else {
            c4 += a_c4;
        }
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

    int32_t* wcount = ws.q_win + n;
    const Sink sink{ws.acc, ws.gid, ws.accG};
    HARP_CK(cudaMemsetAsync(wcount, 0, (size_t)n * sizeof(int32_t), s));
    const size_t small_smem = (size_t)kSmallWarps * kSmallSlots * (sizeof(int32_t) + sizeof(uint32_t));
    HARP_CK(cudaFuncSetAttribute(k_c4_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem));
    k_c4_small<<<152 * 3, kSmallThreads, small_smem, s>>>(ws.off, ws.cols, ws.offp, ws.colsp, ws.deg, ws.dplus,
                                                          ws.fpos, n, warp_max, cta_max, ws.q_mid, ws.q_win, wcount,
                                                          ws.acc, sink);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_SMALL));
    const size_t mid_smem = (size_t)kMidSlots * (sizeof(int32_t) + sizeof(uint32_t));
    HARP_CK(cudaFuncSetAttribute(k_c4_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mid_smem));
    k_c4_mid<<<152, kMidThreads, mid_smem, s>>>(ws.off, ws.cols, ws.offp, ws.colsp, ws.deg, ws.dplus, ws.fpos,
                                                ws.q_mid, n, ws.acc, sink);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_MID));
    HARP_TRY(exclusive_scan_i32_to_i64(wcount, ws.win_prefix, n, ws.scan_tmp, ws.scan_tmp_len, s));
    const size_t win_smem = (size_t)kWinWords * sizeof(uint32_t);
    HARP_CK(cudaFuncSetAttribute(k_c4_window, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem));
    k_c4_window<<<152, kWinThreads, win_smem, s>>>(ws.off, ws.cols, ws.offp, ws.colsp, ws.deg, ws.dplus, ws.fpos,
                                                   n, ws.q_win, ws.win_prefix, ws.acc, sink);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_WINDOW));
    return HARP_OK;
}

}  // namespace harp
