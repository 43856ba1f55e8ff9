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
// cnt(x) <= d-(u).  Rank order sorts each graph's vertices by degree, so inside a graph's rank range
//   * x of degree 1 never complete a cycle: x runs over [n1, u) with n1 the graph's first rank of
//     degree >= 2, and every row's segment starts at fpos[w] (its first neighbour of degree >= 2);
//   * a dense counter for x needs only as many bits as d(x) has, so the x-range splits into bands
//     by degree (d <= 7, 15, 31, 63, 255, 65535, larger) with 3-, 4-, 5-, 6-, 8-, 16- and 32-bit
//     counters packed floor(32 / bits) to a word.  The bands cut into windows of 48-100 KiB of
//     counters form a fixed grid per graph, so the row position of every grid boundary is computed
//     once per row (bpos) instead of being searched for every (root, lower neighbour, window).
// pos_w(u) itself is computed once per lower arc (rev) by a fully parallel pass.
//
// The frontier (the set of x) is not an induced class: whether u ~ x or w1 ~ w2 holds decides
// whether the cycle is induced, a diamond or part of a 4-clique; the closure resolves that mix
// (Section III-C explains why a frontier alone must not be reused as an induced state).
//
// Work per root W(u) = sum_{w in N-(u)} (pos_w(u) - fpos[w]) picks the execution mode:
//   W <= warp_max   one warp, hash table of 1024 slots in shared memory (warp-local mode)
//   W <= mid_max    one warp, hash table of 4096 slots (the middle tier: roots with few wedges spread
//                   over many windows would otherwise cost a whole window pass per window)
//   larger          one block per (root, grid window): dense packed counters in shared memory
//                   (CTA mode); lower neighbours are handed to warps in groups of 32, heaviest first,
//                   and segments of 2048+ elements are split across all warps of the block.  The
//                   window (100, 64 or 48 KiB) sets how many blocks share an SM (2, 3 or 4).
#include <type_traits>

#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int32_t kEmpty = -1;
// Window sizes by resident blocks per SM (plan.c4_window_bytes picks one): 200 KiB for one
// 1024-thread block, 100 KiB at 2 blocks of 512 threads (the default), 64 KiB at 3, 48 KiB at 4
// (counters plus ~3 KiB of static and reserved shared memory per block).  On R-MAT scale 20 the
// 200 KiB window measured 15.7 ms against 13.2 ms for 100 KiB: its fewer (root, window) items do not
// pay for the 32-warp end-of-item barrier there; it is kept for graphs whose x-range spans many windows.
constexpr int kWinWords1 = 51200;
constexpr int kWinWords2 = 25600;
constexpr int kWinWords3 = 16384;
constexpr int kWinWords4 = 12288;
__host__ __device__ constexpr int win_words(int minb) {
    return minb == 1 ? kWinWords1 : (minb == 2 ? kWinWords2 : (minb == 3 ? kWinWords3 : kWinWords4));
}
__host__ __device__ constexpr int win_threads(int minb) { return minb == 1 ? 1024 : 512; }
constexpr int kSmallThreads = 256;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallSlots = 1024;            // per-warp hash table (W <= 512)
constexpr int kMidSlots = 4096;              // per-warp hash table of the middle tier (W <= 2048)
constexpr int kMidWarps = 2;                 // warps per block of the middle tier (64 KiB of tables)
constexpr int kLong = 32;                    // segments this long are read warp-coalesced
constexpr int kSplit = 2048;                 // segments this long are split across the block
constexpr int kSplitQ = 128;                 // split-queue capacity per window item
constexpr int kChunk = 1024;                 // elements per split chunk

// ---------------------------------------------------------------------------------------------
// Per-graph band and grid geometry (ginfo: kGInfo int64 per graph).
// ---------------------------------------------------------------------------------------------
// The window size is a template parameter (WORDS 32-bit words of counters) of every kernel that
// computes window geometry, so each size is its own compiled instance with constant spans.
// The x-range [n1, hi) splits into bands by degree, each with the narrowest counter that is exact
// there (cnt(x) <= d(x) < 2^width): a band of width b packs floor(32 / b) counters into a word.
// ginfo slots: GI_HI, GI_NWIN, then the band starts GI_BAND + b (b = 0 .. kBands - 1; band b
// ends where band b + 1 starts, the last band at GI_HI).  GI_N1 = GI_BAND: the first band starts at n1.
constexpr int kBands = 7;
enum : int { GI_HI = 0, GI_NWIN = 1, GI_BAND = 2, GI_N1 = GI_BAND };
static_assert(GI_BAND + kBands <= kGInfo && kBands < 32, "ginfo slots; one search per lane");

// counter bits of band b and the largest degree the band holds
__host__ __device__ constexpr int band_width(int b) {
    return b == 0 ? 3 : (b == 1 ? 4 : (b == 2 ? 5 : (b == 3 ? 6 : (b == 4 ? 8 : (b == 5 ? 16 : 32)))));
}
__host__ __device__ constexpr int band_per_word(int b) { return 32 / band_width(b); }
__host__ __device__ constexpr int32_t band_max_degree(int b) {
    return band_width(b) >= 31 ? INT32_MAX : (int32_t)((1u << band_width(b)) - 1u);
}

__device__ __forceinline__ int64_t first_above_in(const int32_t* __restrict__ deg, int64_t lo, int64_t hi, int32_t t) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (deg[mid] <= t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// x-values one window of band b covers: the window's words times counters per word
template <int WORDS>
__device__ __forceinline__ int64_t span_of(int b) { return (int64_t)WORDS * band_per_word(b); }

__device__ __forceinline__ int64_t band_end(const int64_t* gi, int b) {
    return b + 1 < kBands ? gi[GI_BAND + b + 1] : gi[GI_HI];
}

// window j of the graph's grid: [xlo, xhi) and its band; false if j is past the grid.  The band loops
// are unrolled, so every span is a compile-time constant.
template <int WORDS>
__device__ __forceinline__ bool grid_window(const int64_t* gi, int64_t j, int64_t& xlo, int64_t& xhi, int& band) {
#pragma unroll
    for (int b = 0; b < kBands; ++b) {
        const int64_t bs = gi[GI_BAND + b], be = band_end(gi, b);
        if (be <= bs) continue;
        const int64_t S = span_of<WORDS>(b);
        const int64_t nb = (be - bs + S - 1) / S;
        if (j < nb) {
            xlo = bs + j * S;
            xhi = xlo + S < be ? xlo + S : be;
            band = b;
            return true;
        }
        j -= nb;
    }
    return false;
}

// number of grid windows that intersect [n1, u)
template <int WORDS>
__device__ __forceinline__ int64_t windows_below(const int64_t* gi, int64_t u) {
    int64_t total = 0;
#pragma unroll
    for (int b = 0; b < kBands; ++b) {
        const int64_t bs = gi[GI_BAND + b], be = band_end(gi, b);
        const int64_t e = be < u ? be : u;
        if (e <= bs) continue;
        const int64_t S = span_of<WORDS>(b);
        total += (e - bs + S - 1) / S;
    }
    return total;
}

// Windows intersecting [n1, u) when bands are merged upwards by mask (bit b set: band b joins band
// b + 1 and takes its wider counters).  st[0 .. kBands] are the unmerged band starts and hi.
template <int WORDS>
__device__ __forceinline__ int64_t merged_windows(const int64_t* st, unsigned mask, int64_t u) {
    int64_t total = 0, gs = st[0];
#pragma unroll
    for (int b = 0; b < kBands; ++b) {
        if (b + 1 < kBands && ((mask >> b) & 1u)) continue;  // the group goes on into band b + 1
        const int64_t e = st[b + 1] < u ? st[b + 1] : u;
        const uint32_t S = (uint32_t)WORDS * (uint32_t)band_per_word(b);  // constant once unrolled
        if (e > gs) total += ((uint32_t)(e - gs) + (S - 1u)) / S;  // ranks and spans fit 31 bits
        gs = st[b + 1];
    }
    return total;
}

constexpr int kMergeMasks = 1 << (kBands - 1);
constexpr int kMergeSamples = 64;

// One warp per graph.  The x-range of a graph's grid is [n1, hi) intersected with [x_lo, x_hi) (a
// partitioned wedge block owns only the opposite vertices in that slice; a whole graph passes
// [0, INT64_MAX)).  A narrow band holding few vertices costs a partly filled window for every root
// that reaches past it, so bands may merge into the next wider one: each lane scores merge masks by
// the windows of kMergeSamples roots spread evenly over the graph's ranks of degree >= 64 (the roots
// that take the windowed mode), each weighted by its degree; the cheapest mask (lowest on a tie) wins.
// merge = false keeps every band separate (mask 0).
template <int WORDS>
__global__ void k_c4_ginfo(const int32_t* __restrict__ deg, int64_t n, const int64_t* __restrict__ gbase,
                           int64_t G, int64_t x_lo, int64_t x_hi, bool merge, int64_t* __restrict__ ginfo) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += warps) {
        const int64_t lo = gbase ? gbase[g] : 0, gend = gbase ? gbase[g + 1] : n;
        auto clamp = [&](int64_t v) { return v < x_lo ? x_lo : (v > x_hi ? x_hi : v); };
        const int64_t hi = gend < x_hi ? gend : x_hi;
        // lane 0: n1 (first rank of degree >= 2); lane b < kBands: the first rank above band b - 1's
        // degrees (band b's start); lane kBands: the first rank of degree >= 64.  One search each.
        const int32_t t = lane == 0 ? 1 : (lane < kBands ? band_max_degree(lane - 1) : 63);
        const int64_t r_lane = lane <= kBands ? first_above_in(deg, lo, gend, t) : gend;
        int64_t n1 = clamp(__shfl_sync(0xffffffffu, r_lane, 0));
        n1 = n1 < hi ? n1 : hi;
        int64_t st[kBands + 1];
        st[0] = n1;
        st[kBands] = hi;
#pragma unroll
        for (int b = 1; b < kBands; ++b) {
            const int64_t r = clamp(__shfl_sync(0xffffffffu, r_lane, b));
            st[b] = r > n1 ? (r < hi ? r : hi) : n1;
        }
        int64_t s0 = __shfl_sync(0xffffffffu, r_lane, kBands);
        if (s0 >= gend) s0 = lo;
        const int64_t span = gend - s0;  // samples u lie in [s0, gend); none for an empty graph
        static_assert(kMergeSamples == 64 && kMergeMasks == 64, "two samples and two masks per lane");
        int64_t us[2];
        double ws[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // lane holds samples lane and lane + 32 (loads issued together)
            us[h] = s0 + (span * (2 * (lane + 32 * h) + 1)) / (2 * kMergeSamples);
            ws[h] = span > 0 ? (double)deg[us[h]] : 0.0;
        }
        unsigned best_mask = 0;  // mask 0: every band separate
        if (merge) {             // uniform over the warp (a kernel argument)
            double best = 0.0;
            for (int m = lane; m < kMergeMasks; m += 32) {
                double c = 0.0;
                for (int k = 0; k < kMergeSamples; ++k) {  // uniform over the warp: every lane shuffles
                    const int64_t u = __shfl_sync(0xffffffffu, k < 32 ? us[0] : us[1], k & 31);
                    const double w = __shfl_sync(0xffffffffu, k < 32 ? ws[0] : ws[1], k & 31);
                    c += w * (double)merged_windows<WORDS>(st, (unsigned)m, u);
                }
                if (m == lane || c < best) {
                    best = c;
                    best_mask = (unsigned)m;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double oc = __shfl_xor_sync(0xffffffffu, best, o);
                const unsigned om = __shfl_xor_sync(0xffffffffu, best_mask, o);
                if (oc < best || (oc == best && om < best_mask)) {
                    best = oc;
                    best_mask = om;
                }
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int b = 0; b + 1 < kBands; ++b)
                if ((best_mask >> b) & 1u) st[b + 1] = st[b];  // band b becomes empty, b + 1 starts at its start
            int64_t* gi = ginfo + g * kGInfo;
            gi[GI_HI] = hi;
#pragma unroll
            for (int b = 0; b < kBands; ++b) gi[GI_BAND + b] = st[b];
            gi[GI_NWIN] = windows_below<WORDS>(gi, hi);
        }
    }
}

// rev[a] = pos_w(u) for every lower arc (u -> w) at position a of u's list.  Each thread takes a run
// of kRevRun consecutive arcs (one search for the run's first row, then it walks forward), so hub
// rows are spread over many threads.  arcs must equal off[n]; the walk never passes row n - 1.
// Whole graph (ROWS = false): the lists are the row prefixes of (off, cols) and the position comes
// from N+(w) (offp, colsp): d-(w) + rank of u in N+(w).  Partitioned (ROWS = true): the lists are
// the roots' lower lists (off = loff, cols = lcols) and the position is searched in w's row of the
// halo (offp = off, colsp = cols of the rows).
constexpr int kRevRun = 16;

template <bool ROWS>
__global__ void __launch_bounds__(256) k_c4_rev(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                                const int64_t* __restrict__ offp, const int32_t* __restrict__ colsp,
                                                const int32_t* __restrict__ deg, const int32_t* __restrict__ dplus,
                                                int64_t n, int64_t arcs, int32_t* __restrict__ rev) {
    const int64_t runs = (arcs + kRevRun - 1) / kRevRun;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < runs; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a0 = r * kRevRun;
        const int64_t a1 = a0 + kRevRun < arcs ? a0 + kRevRun : arcs;
        int64_t lo = 0, hi = n;  // row of arc a0: last u with off[u] <= a0
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= a0) lo = mid;
            else hi = mid;
        }
        int64_t u = lo;
        int64_t ub = off[u], ue = off[u + 1];
        int64_t lower_end = ub + ((int64_t)deg[u] - dplus[u]);
        for (int64_t a = a0; a < a1; ++a) {
            while (a >= ue) {  // next non-empty row
                if (u + 1 >= n) return;  // only if arcs > off[n]
                ++u;
                ub = ue;
                ue = off[u + 1];
                lower_end = ub + ((int64_t)deg[u] - dplus[u]);
            }
            if (a >= lower_end || lower_end - ub < 2) continue;  // only lower arcs of roots with d- >= 2
            const int32_t w = cols[a];
            const int64_t pb = offp[w];
            if (ROWS) rev[a] = (int32_t)lower_bound_i32(colsp + pb, offp[w + 1] - pb, (int32_t)u);
            else rev[a] = (deg[w] - dplus[w]) + (int32_t)lower_bound_i32(colsp + pb, offp[w + 1] - pb, (int32_t)u);
        }
    }
}

// The boundary table keeps kGridCap entries per row: entry k is the row position of grid boundary
// k << s, where s is the smallest shift with ceil((nwin + 1) / 2^s) <= kGridCap (boundary i < nwin is
// the start of window i, boundary nwin the end of the grid).  s = 0 (every boundary) for grids of at
// most kGridCap - 1 windows; larger grids keep every 2^s-th boundary and the rest is found from the
// nearest kept one by a galloping search.
__device__ __forceinline__ int table_shift(int64_t nwin) {
    int sl = 0;
    while (((nwin + 1 + ((int64_t)1 << sl) - 1) >> sl) > kGridCap) ++sl;
    return sl;
}

// First index in [lo, hi) whose element is >= key (a sorted), searching outward from lo: cost grows
// with the log of the distance, not of the row length.
__device__ __forceinline__ int64_t gallop_i32(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t key) {
    if (lo >= hi || __ldg(a + lo) >= key) return lo;
    int64_t prev = lo, step = 1;  // a[prev] < key
    while (prev + step < hi && __ldg(a + prev + step) < key) {
        prev += step;
        step <<= 1;
    }
    int64_t l = prev + 1, r = prev + step < hi ? prev + step : hi;  // the answer lies in [l, r]
    while (l < r) {
        const int64_t mid = (l + r) >> 1;
        if (__ldg(a + mid) < key) l = mid + 1;
        else r = mid;
    }
    return l;
}

// fpos[w] = row position of w's first neighbour of degree >= 2 (the graph's n1 boundary), and
// bpos[w * kGridCap + k] = row position of grid boundary k << s (see table_shift)
template <int WORDS>
__global__ void k_c4_bpos(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                          const int32_t* __restrict__ gid, const int64_t* __restrict__ ginfo, int64_t n,
                          int32_t* __restrict__ fpos, int32_t* __restrict__ bpos) {
    const int64_t total = n * kGridCap;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = t / kGridCap;
        const int k = (int)(t % kGridCap);
        const int64_t* gi = ginfo + (gid ? (int64_t)gid[w] : 0) * kGInfo;
        const int64_t nwin = gi[GI_NWIN];
        if (k == 0) {
            const int64_t wb = off[w];
            const int32_t f = (int32_t)lower_bound_i32(cols + wb, off[w + 1] - wb, (int32_t)gi[GI_N1]);
            fpos[w] = f;
            if (bpos) bpos[t] = f;
            continue;
        }
        const int64_t i = (int64_t)k << table_shift(nwin);
        if (!bpos || i > nwin) continue;
        int64_t bound = gi[GI_HI];
        if (i < nwin) {
            int64_t xhi;
            int band;
            grid_window<WORDS>(gi, i, bound, xhi, band);
        }
        const int64_t wb = off[w];
        bpos[t] = (int32_t)lower_bound_i32(cols + wb, off[w + 1] - wb, (int32_t)bound);
    }
}

// ---------------------------------------------------------------------------------------------
// Segment traversal helpers.  Every loop issues kUnroll independent loads per lane before it uses
// any of them: the per-element work is a load followed by a dependent shared-memory atomic, and
// without the unrolling one load per warp in flight bounds the throughput by latency.
// ---------------------------------------------------------------------------------------------
constexpr int kUnroll = 4;

// Every visitor f(x) returns the previous value of x's counter; the helpers add those values into
// sum.  NARROW: a value fits 16 bits (8- and 16-bit counters, hash counters), so kUnroll of them are
// summed in 32 bits before one 64-bit add.

// Warp-cooperative traversal of 32 segments (lane l owns cols[base_l .. base_l + len_l)):
// flattened so that every lane takes one element per round.
template <bool NARROW, typename F>
__device__ __forceinline__ void warp_flat(const int32_t* __restrict__ cols, int64_t base, int len, F&& f,
                                          uint64_t& sum) {
    const int l = lane_id();
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (l >= o) incl += y;
    }
    const int excl = incl - len;
    const int total = __shfl_sync(kFull, incl, 31);
    for (int t0 = 0; t0 < total; t0 += 32 * kUnroll) {
        int32_t xs[kUnroll];
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
            const int t = t0 + r * 32 + l;
            int o = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int e = __shfl_sync(kFull, excl, o + s);
                if (e <= t) o += s;
            }
            const int64_t ob = __shfl_sync(kFull, base, o);
            const int oe = __shfl_sync(kFull, excl, o);
            xs[r] = t < total ? __ldg(cols + ob + (t - oe)) : 0;
        }
        uint32_t part = 0;
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
            if (t0 + r * 32 + l < total) {
                if (NARROW) part += f(xs[r]);
                else sum += f(xs[r]);
            }
        if (NARROW) sum += part;
    }
}

// n consecutive elements from b, read by the whole warp (coalesced), kUnroll loads in flight per
// lane: whole chunks of 32 * kUnroll without bounds tests, then one guarded tail chunk.
template <bool NARROW, typename F>
__device__ __forceinline__ void warp_run(const int32_t* __restrict__ cols, int64_t b, int n, F&& f, uint64_t& sum) {
    const int l = lane_id();
    const int32_t* __restrict__ p = cols + b + l;
    constexpr int kCh = 32 * kUnroll;
    int k0 = 0;
    for (; k0 + kCh <= n; k0 += kCh) {
        int32_t xs[kUnroll];
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) xs[r] = __ldg(p + k0 + r * 32);
        uint32_t part = 0;
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
            if (NARROW) part += f(xs[r]);
            else sum += f(xs[r]);
        }
        if (NARROW) sum += part;
    }
    if (k0 < n) {
        int32_t xs[kUnroll];
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) xs[r] = k0 + r * 32 + l < n ? __ldg(p + k0 + r * 32) : 0;
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
            if (k0 + r * 32 + l < n) sum += f(xs[r]);
    }
}

// Long segments one after the other, each read by the whole warp (coalesced); short ones flattened.
template <bool NARROW, typename F>
__device__ __forceinline__ void warp_segments(const int32_t* __restrict__ cols, int64_t base, int len, F&& f,
                                              uint64_t& sum) {
    uint32_t longs = __ballot_sync(kFull, len >= kLong);
    while (longs) {
        const int src = __ffs(longs) - 1;
        longs &= longs - 1;
        const int64_t b = __shfl_sync(kFull, base, src);
        const int n = __shfl_sync(kFull, len, src);
        warp_run<NARROW>(cols, b, n, f, sum);
    }
    warp_flat<NARROW>(cols, base, len >= kLong ? 0 : len, f, sum);
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
// Classification: every root (a lane per root, descending rank so heavy roots are queued first).
// ---------------------------------------------------------------------------------------------
template <int WORDS>
__global__ void __launch_bounds__(256) k_c4_classify(const int64_t* __restrict__ loff, const int32_t* __restrict__ lcols,
                                                     const int32_t* __restrict__ deg,
                                                     const int32_t* __restrict__ dplus,
                                                     const int32_t* __restrict__ fpos,
                                                     const int32_t* __restrict__ rev,
                                                     const int32_t* __restrict__ gid,
                                                     const int64_t* __restrict__ ginfo, int64_t n, int64_t own_lo,
                                                     int64_t own_hi, uint32_t warp_max, uint32_t mid_max,
                                                     int32_t* __restrict__ q_small, int32_t* __restrict__ q_win,
                                                     int32_t* __restrict__ wcount, uint64_t* __restrict__ acc) {
    const int l = lane_id();
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long* qcnt_small = (unsigned long long*)&acc[Q_C4_MID];
    unsigned long long* qcnt_mid = (unsigned long long*)&acc[Q_C4_MIDW];
    unsigned long long* qcnt_win = (unsigned long long*)&acc[Q_C4_WIN];
    // a warp takes 32 ranks, one root per lane, spaced by the number of warps (so the hubs at the top
    // ranks fall to different warps): a lane sums W(u) itself when u has at most 32 lower neighbours,
    // the warp sums the larger roots together; queue slots are taken in lane order (descending rank).
    // A warp per root left most lanes idle on the many small roots of a batch of small graphs.
    for (int64_t k0 = wid; k0 < n; k0 += nw * 32) {
        const int64_t k = k0 + (int64_t)l * nw;
        const int32_t u = (int32_t)(n - 1 - k);
        int64_t dm = 0;
        if (k < n && u >= own_lo && u < own_hi) dm = (int64_t)deg[u] - dplus[u];  // the owner rule
        const int64_t ub = dm >= 2 ? loff[u] : 0;
        uint64_t W = 0;
        if (dm >= 2 && dm <= 32) {
            for (int64_t a = 0; a < dm; ++a) {
                const int32_t f = fpos[lcols[ub + a]];
                const int32_t p = rev[ub + a];
                W += p > f ? (uint64_t)(p - f) : 0;
            }
        }
        uint32_t big = __ballot_sync(kFull, dm > 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t bdm = __shfl_sync(kFull, dm, src), bub = __shfl_sync(kFull, ub, src);
            uint64_t bw = 0;
            for (int64_t a = l; a < bdm; a += 32) {
                const int32_t f = fpos[lcols[bub + a]];
                const int32_t p = rev[bub + a];
                bw += p > f ? (uint64_t)(p - f) : 0;
            }
            bw = warp_sum(bw);
            if (l == src) W = bw;
        }
        const int cls = W == 0 ? -1 : (W <= warp_max ? 0 : (W <= mid_max ? 1 : 2));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t mask = __ballot_sync(kFull, cls == c);
            if (!mask) continue;
            unsigned long long base = 0;
            const int leader = __ffs(mask) - 1;
            unsigned long long* ctr = c == 0 ? qcnt_small : (c == 1 ? qcnt_mid : qcnt_win);
            if (l == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
            base = __shfl_sync(kFull, base, leader);
            if (cls == c) {
                const int64_t slot = (int64_t)(base + __popc(mask & lanemask_lt()));
                if (c == 0) {
                    q_small[slot] = u;
                    q_small[n + slot] = (int32_t)W;
                } else if (c == 1) {  // the middle tier fills the same queue from the back
                    q_small[n - 1 - slot] = u;
                    q_small[2 * n - 1 - slot] = (int32_t)W;
                } else {
                    const int64_t* gi = ginfo + (gid ? (int64_t)gid[u] : 0) * kGInfo;
                    q_win[slot] = u;
                    wcount[slot] = (int32_t)windows_below<WORDS>(gi, u);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Warp-local mode: one warp per queued small root, hash table in shared memory.
// ---------------------------------------------------------------------------------------------
// SLOTS hash slots per warp, WARPS warps per block; MID: the middle tier's queue (from the back of
// q_small, length acc[Q_C4_MIDW]) instead of the warp-local one (from the front, acc[Q_C4_MID]).
template <int SLOTS, int WARPS, bool MID>
__global__ void __launch_bounds__(WARPS * 32, 3) k_c4_small(const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ cols,
                                                            const int64_t* __restrict__ loff,
                                                            const int32_t* __restrict__ lcols,
                                                            const int32_t* __restrict__ deg,
                                                            const int32_t* __restrict__ dplus,
                                                            const int32_t* __restrict__ fpos,
                                                            const int32_t* __restrict__ rev,
                                                            const int32_t* __restrict__ q_small, int64_t n,
                                                            uint64_t* __restrict__ acc, Sink sink) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* my_keys = reinterpret_cast<int32_t*>(smem_raw) + (threadIdx.x >> 5) * SLOTS;
    uint32_t* my_cnt = reinterpret_cast<uint32_t*>(smem_raw + WARPS * SLOTS * sizeof(int32_t)) +
                       (threadIdx.x >> 5) * SLOTS;
    __shared__ uint64_t red[32];
    const int l = lane_id();
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nq = (int64_t)acc[MID ? Q_C4_MIDW : Q_C4_MID];
    uint64_t c4 = 0;
    for (int64_t k = wid; k < nq; k += nw) {
        const int64_t slot = MID ? n - 1 - k : k;
        const int32_t u = q_small[slot];
        const uint32_t W = (uint32_t)q_small[n + slot];
        const int64_t dm = (int64_t)deg[u] - dplus[u];
        const int64_t ub = loff[u];
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
                const int32_t wv = lcols[ub + a];
                const int32_t f = fpos[wv];
                const int32_t p = rev[ub + a];
                base = off[wv] + f;
                len = p > f ? p - f : 0;
            }
            warp_flat<true>(cols, base, len, [&](int32_t x) { return hash_add(my_keys, my_cnt, P - 1, x); }, a_c4);
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
// Windowed CTA mode: one block per (root, grid window); dense packed counters in shared memory.
// ---------------------------------------------------------------------------------------------
// Packed counters: a band of width b packs floor(32 / b) counters into a word (3-bit ten, 4-bit
// eight, 5-bit six, 6-bit five, 8-bit four, 16-bit two).  (A byte-plane layout that
// puts consecutive x in consecutive banks was measured no faster: the kernel is bound by load
// latency and the end-of-item barrier, not by shared-memory bank conflicts.)
template <int WIDTH, int WORDS>
__device__ __forceinline__ uint32_t counter_add(uint32_t* cw, uint32_t r) {
    constexpr uint32_t K = 32 / WIDTH;  // counters per word
    if constexpr (K == 1) {
        return atomicAdd(&cw[r], 1u);
    } else {
        const uint32_t q = r / K;  // a constant divisor: a multiply and a shift
        const uint32_t sh = (r - q * K) * WIDTH;
        return (atomicAdd(&cw[q], 1u << sh) >> sh) & ((1u << WIDTH) - 1u);
    }
}

// Calls f(std::integral_constant<int, width>) for band b's counter width, so each width is its own
// compiled instance of the window and split passes.
template <typename F>
__device__ __forceinline__ void with_band(int b, F&& f) {
    switch (b) {
        case 0: f(std::integral_constant<int, band_width(0)>{}); break;
        case 1: f(std::integral_constant<int, band_width(1)>{}); break;
        case 2: f(std::integral_constant<int, band_width(2)>{}); break;
        case 3: f(std::integral_constant<int, band_width(3)>{}); break;
        case 4: f(std::integral_constant<int, band_width(4)>{}); break;
        case 5: f(std::integral_constant<int, band_width(5)>{}); break;
        default: f(std::integral_constant<int, band_width(6)>{}); break;
    }
}
static_assert(kBands == 7, "with_band covers every band");

struct WinShared {
    int group;                 // next group of 32 lower neighbours
    int nsplit;                // entries pushed to the split queue
    int chunk;                 // next split chunk
    int64_t split_base[kSplitQ];
    int32_t split_len[kSplitQ];
    int32_t split_pre[kSplitQ + 1];
};

// Self-check: a segment outside its row, or one whose first or last element lies outside the window
// (rows are sorted, so these two bound every element of the segment), is skipped and recorded in
// acc[ACC_ERR]; the host then reports HARP_EDEVICE.
__device__ __forceinline__ void flag_error(uint64_t* acc, unsigned long long bit) {
    atomicOr((unsigned long long*)&acc[ACC_ERR], bit);
}

template <int WIDTH, int WORDS>
__device__ __forceinline__ void window_pass(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                            const int32_t* __restrict__ lcols,
                                            const int32_t* __restrict__ fpos, const int32_t* __restrict__ rev,
                                            const int32_t* __restrict__ bpos, bool table, int sl, int64_t nwin,
                                            int64_t j, int64_t ub,
                                            int64_t dm, int32_t xlo, int32_t xhi, bool first, bool last, uint32_t* cw,
                                            WinShared& sh, uint64_t& c4, uint64_t* acc) {
    const int l = lane_id();
    auto add = [&](int32_t x) { return counter_add<WIDTH, WORDS>(cw, (uint32_t)(x - xlo)); };
    const int ngroups = (int)((dm + 31) >> 5);
    for (;;) {
        int g = 0;
        if (l == 0) g = atomicAdd(&sh.group, 1);
        g = __shfl_sync(kFull, g, 0);
        if (g >= ngroups) break;
        const int64_t a = (int64_t)(ngroups - 1 - g) * 32 + l;  // heaviest groups first
        int64_t base = 0;
        int len = 0;
        if (a < dm) {
            const int32_t wv = lcols[ub + a];
            const int64_t wb = off[wv];
            int64_t p0, p1;
            const int64_t rowlen = off[wv + 1] - wb;
            const int64_t mask = ((int64_t)1 << sl) - 1;
            if (first) p0 = fpos[wv];
            else if (table && (j & mask) == 0) p0 = bpos[(int64_t)wv * kGridCap + (j >> sl)];
            else if (table) p0 = gallop_i32(cols + wb, bpos[(int64_t)wv * kGridCap + (j >> sl)], rowlen, xlo);
            else p0 = lower_bound_i32(cols + wb, rowlen, xlo);
            if (last) p1 = rev[ub + a];
            else if (table && ((j + 1) & mask) == 0 && j + 1 <= nwin) p1 = bpos[(int64_t)wv * kGridCap + ((j + 1) >> sl)];
            else if (table) p1 = gallop_i32(cols + wb, p0 < 0 ? 0 : p0, rowlen, xhi);
            else p1 = lower_bound_i32(cols + wb, rowlen, xhi);
            if (p0 < 0 || p1 > rowlen) {
                flag_error(acc, kErrRow);
                p0 = p1 = 0;
            }
            if (p1 > p0 && (cols[wb + p0] < xlo || cols[wb + p1 - 1] >= xhi)) {
                flag_error(acc, kErrSegment);
                p1 = p0;
            }
            base = wb + p0;
            len = p1 > p0 ? (int)(p1 - p0) : 0;
        }
        if (len >= kSplit) {  // hand very long segments to the whole block
            const int slot = atomicAdd(&sh.nsplit, 1);
            if (slot < kSplitQ) {
                sh.split_base[slot] = base;
                sh.split_len[slot] = len;
                len = 0;
            }
        }
        warp_segments<WIDTH != 32>(cols, base, len, add, c4);
    }
}

template <int WIDTH, int WORDS>
__device__ __forceinline__ void split_pass(const int32_t* __restrict__ cols, int32_t xlo, uint32_t* cw, WinShared& sh,
                                           uint64_t& c4) {
    const int l = lane_id();
    const int ns = sh.nsplit < kSplitQ ? sh.nsplit : kSplitQ;
    const int total = sh.split_pre[ns];
    for (;;) {
        int t = 0;
        if (l == 0) t = atomicAdd(&sh.chunk, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= total) break;
        int e = 0;  // entry owning chunk t: last e with split_pre[e] <= t
        int hi = ns;
        while (hi - e > 1) {
            const int mid = (e + hi) >> 1;
            if (sh.split_pre[mid] <= t) e = mid;
            else hi = mid;
        }
        const int64_t b = sh.split_base[e] + (int64_t)(t - sh.split_pre[e]) * kChunk;
        const int64_t end = sh.split_base[e] + sh.split_len[e];
        const int64_t stop = b + kChunk < end ? b + kChunk : end;
        warp_run<WIDTH != 32>(cols, b, (int)(stop - b),
                              [&](int32_t x) { return counter_add<WIDTH, WORDS>(cw, (uint32_t)(x - xlo)); }, c4);
    }
}

// Everything an item (root, grid window) needs before its lower neighbours are walked.  Resolving it
// is a chain of dependent loads (ticket, search of the item's root, the root, its grid window, its
// list), so one thread resolves the next item while the block works on the current one.
struct WinItem {
    int64_t t;  // ticket; >= the item total: no more items
    int64_t j, xlo, xhi, nwin, dm, ub;
    int32_t u;
    int band, sl, first, last;
};

template <int WORDS>
__device__ __forceinline__ void resolve_item(WinItem& it, int64_t t, int64_t total, int64_t nroots,
                                             const int64_t* __restrict__ win_prefix,
                                             const int32_t* __restrict__ q_win, const int32_t* __restrict__ gid,
                                             const int64_t* __restrict__ ginfo, const int32_t* __restrict__ deg,
                                             const int32_t* __restrict__ dplus, const int64_t* __restrict__ loff) {
    it.t = t;
    if (t >= total) return;
    int64_t lo = 0, hi = nroots;  // root index: last k with win_prefix[k] <= t
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (win_prefix[mid] <= t) lo = mid;
        else hi = mid;
    }
    const int32_t u = q_win[lo];
    const int64_t j = t - win_prefix[lo];
    const int64_t* gi = ginfo + (gid ? (int64_t)gid[u] : 0) * kGInfo;
    int64_t xlo = 0, xhi = 0;
    int band = kBands - 1;
    grid_window<WORDS>(gi, j, xlo, xhi, band);
    it.last = xhi >= (int64_t)u;
    it.xhi = it.last ? u : xhi;
    it.xlo = xlo;
    it.first = j == 0;
    it.j = j;
    it.u = u;
    it.band = band;
    it.nwin = gi[GI_NWIN];
    it.sl = table_shift(it.nwin);
    it.dm = (int64_t)deg[u] - dplus[u];
    it.ub = loff[u];
}

template <int MINB>
__global__ void __launch_bounds__(win_threads(MINB), MINB) k_c4_window(const int64_t* __restrict__ off,
                                                              const int32_t* __restrict__ cols,
                                                              const int64_t* __restrict__ loff,
                                                              const int32_t* __restrict__ lcols,
                                                              const int32_t* __restrict__ deg,
                                                              const int32_t* __restrict__ dplus,
                                                              const int32_t* __restrict__ fpos,
                                                              const int32_t* __restrict__ rev,
                                                              const int32_t* __restrict__ bpos,
                                                              const int32_t* __restrict__ gid,
                                                              const int64_t* __restrict__ ginfo,
                                                              const int32_t* __restrict__ q_win,
                                                              const int64_t* __restrict__ win_prefix,
                                                              uint64_t* __restrict__ acc, Sink sink) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* cw = reinterpret_cast<uint32_t*>(smem_raw);
    constexpr int WORDS = win_words(MINB);
    __shared__ WinItem s_next;
    __shared__ WinShared sh;
    __shared__ uint64_t red[32];
    const int64_t nroots = (int64_t)acc[Q_C4_WIN];
    const int64_t total = win_prefix[nroots];
    unsigned long long* ticket = (unsigned long long*)&acc[T_C4_WIN];
    const bool table = bpos != nullptr;
    uint64_t c4 = 0;
    if (threadIdx.x == 0)
        resolve_item<WORDS>(s_next, (int64_t)atomicAdd(ticket, 1ull), total, nroots, win_prefix, q_win, gid, ginfo,
                            deg, dplus, loff);
    __syncthreads();
    for (;;) {
        const WinItem it = s_next;
        if (it.t >= total) break;
        const int32_t u = it.u;
        const int64_t j = it.j, xlo = it.xlo, xhi = it.xhi, nwin = it.nwin, dm = it.dm, ub = it.ub;
        const int band = it.band, sl = it.sl;
        const bool first = it.first, last = it.last;
        if (threadIdx.x == 0) {
            sh.group = 0;
            sh.nsplit = 0;
            sh.chunk = 0;
        }
        int words = 0;
        with_band(band, [&](auto wc) {
            constexpr int per = 32 / decltype(wc)::value;
            words = (int)((xhi - xlo + per - 1) / per);
        });
        for (int i = threadIdx.x; i < words; i += win_threads(MINB)) cw[i] = 0;
        __syncthreads();  // every thread holds this item; counters and work counters are reset
        if (threadIdx.x == 0)  // the next item, resolved while the block walks this one
            resolve_item<WORDS>(s_next, (int64_t)atomicAdd(ticket, 1ull), total, nroots, win_prefix, q_win, gid,
                                ginfo, deg, dplus, loff);
        uint64_t a_c4 = 0;
        with_band(band, [&](auto wc) {
            window_pass<decltype(wc)::value, WORDS>(off, cols, lcols, fpos, rev, bpos, table, sl, nwin, j, ub, dm,
                                                    (int32_t)xlo, (int32_t)xhi, first, last, cw, sh, a_c4, acc);
        });
        __syncthreads();
        if (sh.nsplit > 0) {
            if (threadIdx.x == 0) {
                const int ns = sh.nsplit < kSplitQ ? sh.nsplit : kSplitQ;
                int run = 0;
                for (int e = 0; e < ns; ++e) {
                    sh.split_pre[e] = run;
                    run += (sh.split_len[e] + kChunk - 1) / kChunk;
                }
                sh.split_pre[ns] = run;
            }
            __syncthreads();
            with_band(band, [&](auto wc) { split_pass<decltype(wc)::value, WORDS>(cols, (int32_t)xlo, cw, sh, a_c4); });
            __syncthreads();
        }
        if (sink.batch()) {
            const uint64_t s = block_sum_u64(a_c4, red);
            if (threadIdx.x == 0) sink_add(sink, u, G_C4, s);
        } else {
            c4 += a_c4;
        }
        __syncthreads();  // every thread is done with this item's shared state; s_next is resolved
    }
    c4 = block_sum_u64(c4, red);
    if (threadIdx.x == 0 && c4) atomicAdd((unsigned long long*)&acc[ACC_C4], (unsigned long long)c4);
}

unsigned grid_cap(int64_t work, int threads, int64_t cap) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// The whole wedge pass for one window size (MINB resident window blocks per SM).
template <int MINB>
harp_status wedge_pass(const harp_csr* g, Workspace& ws, uint32_t warp_max, uint32_t mid_max, bool merge,
                       cudaStream_t s) {
    constexpr int WORDS = win_words(MINB);
    const int64_t n = g->n;
    const int64_t G = ws.G > 0 ? ws.G : 1;
    const Sink sink{ws.acc, ws.gid, ws.accG};
    const int sms = num_sms();
    int32_t* wcount = ws.q_win + n;
    HARP_CK(cudaMemsetAsync(wcount, 0, (size_t)n * sizeof(int32_t), s));
    k_c4_ginfo<WORDS><<<grid_cap(G * 32, 128, 1024), 128, 0, s>>>(ws.deg, n, ws.gbase, G, ws.x_lo, ws.x_hi, merge,
                                                                  ws.ginfo);
    HARP_LAUNCHED();
    // the roots' lower lists: row prefixes of a whole graph, or their own CSR in a partitioned block
    const bool lists = ws.loff != nullptr;
    const int64_t* loff = lists ? ws.loff : ws.off;
    const int32_t* lcols = lists ? ws.lcols : ws.cols;
    if (lists) {
        const int64_t la = ws.lower_arcs;  // == loff[n]
        k_c4_rev<true><<<grid_cap((la + kRevRun - 1) / kRevRun, 256, (int64_t)sms * 64), 256, 0, s>>>(
            ws.loff, ws.lcols, ws.off, ws.cols, ws.deg, ws.dplus, n, la, ws.rev);
    } else {
        const int64_t arcs = ws.arcs >= 0 ? ws.arcs : 2 * g->m;  // must equal off[n]
        k_c4_rev<false><<<grid_cap((arcs + kRevRun - 1) / kRevRun, 256, (int64_t)sms * 64), 256, 0, s>>>(
            ws.off, ws.cols, ws.offp, ws.colsp, ws.deg, ws.dplus, n, arcs, ws.rev);
    }
    HARP_LAUNCHED();
    k_c4_bpos<WORDS><<<grid_cap(n * kGridCap, 256, (int64_t)sms * 64), 256, 0, s>>>(ws.off, ws.cols, ws.gid, ws.ginfo, n,
                                                                             ws.fpos, ws.bpos);
    HARP_LAUNCHED();
    k_c4_classify<WORDS><<<grid_cap(n, 256, (int64_t)sms * 32), 256, 0, s>>>(  // a lane per root
        loff, lcols, ws.deg, ws.dplus, ws.fpos, ws.rev, ws.gid, ws.ginfo, n, ws.own_lo, ws.own_hi, warp_max,
        mid_max, ws.q_mid, ws.q_win, wcount, ws.acc);
    HARP_LAUNCHED();
    const size_t small_smem = (size_t)kSmallWarps * kSmallSlots * (sizeof(int32_t) + sizeof(uint32_t));
    HARP_CK(cudaFuncSetAttribute(k_c4_small<kSmallSlots, kSmallWarps, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem));
    k_c4_small<kSmallSlots, kSmallWarps, false><<<sms * 3, kSmallThreads, small_smem, s>>>(
        ws.off, ws.cols, loff, lcols, ws.deg, ws.dplus, ws.fpos, ws.rev, ws.q_mid, n, ws.acc, sink);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_SMALL));
    if (mid_max > warp_max) {  // the middle tier: 4096-slot warp tables, three 2-warp blocks per SM
        const size_t mid_smem = (size_t)kMidWarps * kMidSlots * (sizeof(int32_t) + sizeof(uint32_t));
        HARP_CK(cudaFuncSetAttribute(k_c4_small<kMidSlots, kMidWarps, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mid_smem));
        k_c4_small<kMidSlots, kMidWarps, true><<<sms * 3, kMidWarps * 32, mid_smem, s>>>(
            ws.off, ws.cols, loff, lcols, ws.deg, ws.dplus, ws.fpos, ws.rev, ws.q_mid, n, ws.acc, sink);
        HARP_LAUNCHED();
    }
    HARP_CK(prof_mark(s, SEG_C4_MID));
    HARP_TRY(exclusive_scan_i32_to_i64(wcount, ws.win_prefix, n, ws.scan_tmp, ws.scan_tmp_len, s));
    const size_t win_smem = (size_t)WORDS * sizeof(uint32_t);
    HARP_CK(cudaFuncSetAttribute(k_c4_window<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem));
    k_c4_window<MINB><<<sms * MINB, win_threads(MINB), win_smem, s>>>(ws.off, ws.cols, loff, lcols, ws.deg, ws.dplus,
                                                                ws.fpos, ws.rev,
                                                                ws.bpos, ws.gid, ws.ginfo, ws.q_win, ws.win_prefix,
                                                                ws.acc, sink);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_C4_WINDOW));
    return HARP_OK;
}

}  // namespace

harp_status count_wedge_c4(const harp_csr* g, Workspace& ws, const harp_plan& plan, cudaStream_t s) {
    if (g->n == 0 || g->m == 0) return HARP_OK;
    uint32_t warp_max = plan.c4_warp_max_work ? plan.c4_warp_max_work : 512;
    if (warp_max > kSmallSlots / 2) warp_max = kSmallSlots / 2;
    // the middle tier takes kMidSlots / 2 wedges at most; c4_cta_max_work <= warp_max turns it off
    uint32_t mid_max = plan.c4_cta_max_work;
    if (mid_max > kMidSlots / 2) mid_max = kMidSlots / 2;
    if (mid_max < warp_max) mid_max = warp_max;
    // window size: the largest of the four that fits plan.c4_window_bytes (at least the smallest).
    // 0 = by graph: a single graph of more than 2^22 vertices takes 200 KiB (its x-range spans tens to
    // hundreds of 100 KiB windows, and halving the (root, window) visits measured 37.7 -> 26.1 s on
    // the 5e7-vertex Chung-Lu graph), anything smaller and every batch 100 KiB (R-MAT scale 20: 13.2
    // ms at 100 KiB against 15.7 ms at 200 KiB)
    const bool merge = !(plan.flags & HARP_PLAN_NO_BAND_MERGE);
    uint32_t wbytes = plan.c4_window_bytes;
    if (wbytes == 0) wbytes = (ws.G <= 1 && g->n > ((int64_t)1 << 22)) ? (uint32_t)kWinWords1 * 4 : (uint32_t)kWinWords2 * 4;
    if (wbytes >= (uint32_t)kWinWords1 * 4) return wedge_pass<1>(g, ws, warp_max, mid_max, merge, s);
    if (wbytes >= (uint32_t)kWinWords2 * 4) return wedge_pass<2>(g, ws, warp_max, mid_max, merge, s);
    if (wbytes >= (uint32_t)kWinWords3 * 4) return wedge_pass<3>(g, ws, warp_max, mid_max, merge, s);
    return wedge_pass<4>(g, ws, warp_max, mid_max, merge, s);
}

}  // namespace harp
