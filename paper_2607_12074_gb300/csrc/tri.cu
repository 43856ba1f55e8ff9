// Steps a3 + a4: triangle anchors with per-edge triangle statistics, and their 4-clique extension
// (Section III-B: "for 4-node motifs, anchors include ordered wedges and triangles"; Section III-F:
// X_3 / 4-cliques; Section III-D: warp-local vs CTA mode, ordered set intersection, compaction,
// block-local aggregation).
//
// In rank order every triangle {u < v < w} is anchored once at its lowest vertex u.  For an anchor
// vertex u with out-neighbourhood L = N+(u) (sorted, d = |L|) we build the oriented adjacency of
// G[L] as a bitmap: row i has bit j (j > i) iff L[j] is in N+(L[i]).  Row i is the candidate
// frontier of the partial embedding (u, L[i]) (its signature: j = 2, frontier generator (u, L[i]),
// required adjacency to both, no forbidden edge); it is computed once by an ordered intersection of
// N+(L[i]) with L and then reused for
//   * triangles:   T_u = sum_i popc(row_i)
//   * t_e:         arc (u, L[i]) gets popc(row_i) + (# rows with bit i); arc (L[i], L[j]) gets +1
//                  per set bit (global atomic at the position where the intersection found it)
//   * 4-cliques:   K4_u = sum over set bits (i, j) of popc(row_i & row_j)   (the X_3 extension)
//   * paw sums:    sum over triangles of (d_a + d_b + d_c)
// The intersection either probes the exact range of N+(L[i]) in [L[i+1], max L] (16-byte loads, a
// membership filter while hits are rare, then the index j of each element in L), or, where few keys
// of L remain after L[i], searches each of those keys in N+(L[i]) (row_searches).
// Warp-local mode: d <= tri_warp_max (<= 32), rows are single words, one warp per anchor.
// CTA mode: up to tri_cta_max (<= 1024) in three sizes (256 / 512 / 1024), rows in shared memory, one
// block per anchor; the 4-clique sum is dealt to the block as (word, row) units of the bitmap.  Global-staged mode (up to tri_big_max <= 4096, hubs of very large skewed
// graphs): the same rows in a per-block scratch that stays in L2 (d^2 / 8 bytes), each row built in
// a per-warp shared buffer and written out once.  Fallback (larger d): per out-arc ordered
// intersections through global memory with binary-searched membership; 4-cliques by binary search
// in N+(w).  Membership of y in L is a hash lookup (HARP_PROBE_HASH) or a binary search of the
// sorted L in shared memory (HARP_PROBE_BSEARCH); with the hash, a CTA anchor whose L spans few ranks
// uses a direct table indexed by y - L[0] in the hash's bytes instead.
//
// Signature reuse (Section III-C): the extension of (u, v, w) to a 4-clique needs
// |N+(w) n S_uv|, and since S_uv is a subset of L this is popc(row_v & row_w): the staged frontier of
// the signature (u, w) answers it.  Every triangle is one such lookup; it is a hit when the anchor's
// rows are staged (warp and CTA modes) and a miss in the fallback, which recomputes the
// intersection from N+(w).  With reuse switched off (HARP_PLAN_NO_REUSE) the staged modes recompute
// too, by walking N+(w) in global memory; the counts are identical either way.  acc[ACC_SIG_HITS]
// counts hits; the lookups are the triangles.
#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kCta1 = 256;
// Block shape of the 256 mode: 192 threads, 7 resident blocks per SM (48 registers a thread).  On
// R-MAT scale 20 it measured 5.49 ms against 5.77 ms for 256 x 5 and 6.09 ms for 128 x 9: an anchor's
// rows spread over fewer warps wait less at its block barriers, and more blocks share each SM.
constexpr int kCta1Threads = 192;
constexpr int kCta1Blocks = 7;
constexpr int kCta2 = 512;
constexpr int kCtaMax = 1024;
constexpr int kInf = 0x7fffffff;
constexpr int32_t kNoKey = -1;

// Anchor queues: in ws.q_tri (n entries) warp-mode anchors (2 <= d <= tri_warp_max) from the front
// and CTA-mode anchors from the back; fallback anchors in ws.q_mid[0, n) and global-staged anchors in
// ws.q_mid[n, 2n) (q_mid is free until the wedge pass).  Vertices are scanned in descending rank, so high-degree anchors tend to be queued
// (and taken) first.
//
// Tier of an anchor of out-degree d: -1 none, 0 warp, 1/2/3 CTA 256/512/1024, 4 global-staged,
// 5 fallback.  wmax <= 32, cmax <= kCtaMax, bmax <= kBigMax (tri_warp_max / tri_cta_max / tri_big_max).
constexpr int kBigMax = 4096;
__device__ __forceinline__ int tri_class(int d, int wmax, int cmax, int bmax) {
    if (d < 2) return -1;
    if (d <= wmax) return 0;
    if (d > cmax) return d <= bmax ? 4 : 5;
    return d <= kCta1 ? 1 : (d <= kCta2 ? 2 : 3);
}

__global__ void k_tri_classify(const int32_t* __restrict__ dplus, int64_t n, int64_t own_lo, int64_t own_hi,
                               int wmax, int cmax, int bmax, int32_t* __restrict__ q, int32_t* __restrict__ q_fb,
                               unsigned long long* __restrict__ cnt, unsigned long long* __restrict__ cnt_fb,
                               unsigned long long* __restrict__ cnt_big) {
    const int l = lane_id();
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - l; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = n - 1 - (base + l);
        int cls = -1;
        if (u >= own_lo && u < own_hi && u < n) cls = tri_class(dplus[u], wmax, cmax, bmax);
        // 0: warp queue, 1: CTA queue, 2: fallback queue, 3: global-staged queue
        cls = cls == 5 ? 2 : (cls == 4 ? 3 : (cls > 0 ? 1 : cls));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t mask = __ballot_sync(kFull, cls == c);
            if (!mask) continue;
            unsigned long long start = 0;
            const int leader = __ffs(mask) - 1;
            unsigned long long* ctr = c < 2 ? &cnt[c] : (c == 2 ? cnt_fb : cnt_big);
            if (l == leader) start = atomicAdd(ctr, (unsigned long long)__popc(mask));
            start = __shfl_sync(kFull, start, leader);
            if (cls == c) {
                const unsigned long long k = start + __popc(mask & lanemask_lt());
                if (c == 0) q[k] = (int32_t)u;
                else if (c == 1) q[n - 1 - (int64_t)k] = (int32_t)u;
                else if (c == 2) q_fb[k] = (int32_t)u;
                else q_fb[n + (int64_t)k] = (int32_t)u;
            }
        }
    }
}

// Shared-memory hash of the anchor list: key = vertex, value = its index in L.  2^bits slots.
template <typename V>
__device__ __forceinline__ void hash_put(int32_t* hk, V* hv, int bits, int32_t key, int idx) {
    const uint32_t mask = (1u << bits) - 1;
    uint32_t h = hash32((uint32_t)key) >> (32 - bits);
    for (;;) {
        if (atomicCAS(&hk[h], kNoKey, key) == kNoKey) {
            hv[h] = (V)idx;
            return;
        }
        h = (h + 1) & mask;
    }
}

template <typename V>
__device__ __forceinline__ int hash_get(const int32_t* hk, const V* hv, int bits, int32_t key) {
    const uint32_t mask = (1u << bits) - 1;
    uint32_t h = hash32((uint32_t)key) >> (32 - bits);
    for (;;) {
        const int32_t k = hk[h];
        if (k == key) return (int)hv[h];
        if (k == kNoKey) return -1;
        h = (h + 1) & mask;
    }
}

// Index of y in the sorted list L[0, d) (shared memory), or -1.
__device__ __forceinline__ int find_sorted(const int32_t* L, int d, int32_t y) {
    int lo = 0, hi = d;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (L[mid] < y) lo = mid + 1;
        else hi = mid;
    }
    return (lo < d && L[lo] == y) ? lo : -1;
}

// First position p in [lo, hi) with a[p] >= t, found by the whole warp (32-ary search).
__device__ __forceinline__ int64_t warp_lower_bound(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t t) {
    const int l = lane_id();
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t idx = lo + (int64_t)(l + 1) * step - 1;
        const bool pred = idx >= hi || a[idx] >= t;
        const uint32_t m = __ballot_sync(kFull, pred);
        if (!m) return hi;  // every probed element (the last one included) is below t
        const int k = __ffs(m) - 1;
        const int64_t nlo = lo + (int64_t)k * step;
        const int64_t nhi = nlo + step < hi ? nlo + step : hi;
        lo = nlo;
        hi = nhi;
    }
    const bool pred = lo + l < hi && a[lo + l] >= t;
    const uint32_t m = __ballot_sync(kFull, pred);
    return m ? lo + __ffs(m) - 1 : hi;
}

// Walk the sorted list colsp[b, e) in warp-wide chunks with kProbeUnroll chunks' loads in flight,
// calling probe(y, position) for every element, and stop after the chunk that passes `last`.
constexpr int kProbeUnroll = 2;

template <typename F>
__device__ __forceinline__ void probe_list(const int32_t* __restrict__ colsp, int64_t b, int64_t e, int32_t last,
                                           F&& probe) {
    const int l = lane_id();
    for (int64_t p0 = b; p0 < e; p0 += 32 * kProbeUnroll) {
        int32_t ys[kProbeUnroll];
#pragma unroll
        for (int r = 0; r < kProbeUnroll; ++r) {
            const int64_t p = p0 + r * 32 + l;
            ys[r] = p < e ? colsp[p] : kInf;
        }
        bool done = false;
#pragma unroll
        for (int r = 0; r < kProbeUnroll; ++r) {
            if (!done) {
                probe(ys[r], p0 + r * 32 + l);
                done = __shfl_sync(kFull, ys[r], 31) >= last;  // rows are sorted: past the largest candidate
            }
        }
        if (done) break;
    }
}

// Probe every element of colsp[b, e) (an exact range) with 16-byte loads.  The range is widened to
// 4-element boundaries: colsp starts on a 256-byte boundary and its allocation is padded to a multiple
// of 256 bytes, so the wider loads stay inside it; lane l takes elements a + 128 k + 4 l .. + 3 (a = b
// rounded down to a multiple of 4) and masks those outside [b, e).  visit(y, p) gets the element and
// its position in colsp.
// With `filter` (warp-uniform) the membership test may_hold(y) (a filter bit: 0 proves y absent) runs
// first on all four elements and the lane then visits only those that pass, so 128 elements pay for
// the divergent lookup and hit paths once per candidate of the busiest lane, instead of once per 32
// elements whenever any lane holds a candidate.  Without it (rows where hits are common) every
// element is visited.
template <typename Filter, typename Visit>
__device__ __forceinline__ void probe_filtered(const int32_t* __restrict__ colsp, int64_t b, int64_t e, bool filter,
                                               Filter&& may_hold, Visit&& visit) {
    const int64_t a = b & ~(int64_t)3;
    const int4* __restrict__ v = reinterpret_cast<const int4*>(colsp + a);
    const int lo = (int)(b - a), hi = (int)(e - a);  // the range's offsets from a: lo <= 3
    for (int q = 4 * lane_id(); q < hi; q += 128) {
        const int4 y = __ldg(v + (q >> 2));
        uint32_t valid = hi - q >= 4 ? 0xfu : (1u << (hi - q)) - 1u;
        if (q < lo) valid &= 0xfu << (lo - q);
        if (filter) {
            uint32_t cand = may_hold(y.x) | (may_hold(y.y) << 1) | (may_hold(y.z) << 2) | (may_hold(y.w) << 3);
            cand &= valid;
            while (cand) {
                const int r = __ffs(cand) - 1;
                cand &= cand - 1;
                const int32_t x = r == 0 ? y.x : (r == 1 ? y.y : (r == 2 ? y.z : y.w));
                visit(x, a + q + r);
            }
        } else {
            if (valid & 1u) visit(y.x, a + q);
            if (valid & 2u) visit(y.y, a + q + 1);
            if (valid & 4u) visit(y.z, a + q + 2);
            if (valid & 8u) visit(y.w, a + q + 3);
        }
    }
}

// Whether the next row is probed through the membership filter: the filter pays while hits are rare.
// Each warp keeps its own probe and hit totals over the rows it has taken (halved past 2^20 probes, so
// they follow the current anchors) and filters while fewer than one probe in eight has hit.
struct FilterChoice {
    uint32_t probes = 0, hits = 0;
    __device__ __forceinline__ bool use() const { return 8u * hits <= probes; }
    __device__ __forceinline__ void add(int64_t row_probes, uint32_t row_hits) {
        probes += (uint32_t)row_probes;
        hits += row_hits;
        if (probes > (1u << 20)) {
            probes >>= 1;
            hits >>= 1;
        }
    }
};

// Row i's hits can be found from either side: probe every element of its range (one load and a
// filter or hash lookup each), or search each of the keys of L left after L[i] in the range (a binary
// search of about log2(len) + 1 dependent loads each, which the row's few cache lines keep in L1).
// Searching costs less when keys * (log2(len) + 1) < 2 * len: rows near the end of L and rows of long
// ranges.  Both find exactly the members of L in the range.
__device__ __forceinline__ bool row_searches(int keys, int64_t len) {
    if (len <= 0) return false;  // no element: nothing to do either way
    const int lg = 64 - __clzll(len);  // floor(log2(len)) + 1
    return (int64_t)keys * lg < 2 * len;
}

// Position of key in the sorted colsp[b, b + len), or -1.
__device__ __forceinline__ int64_t find_in_range(const int32_t* __restrict__ colsp, int64_t b, int len, int32_t key) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(colsp + b + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < len && __ldg(colsp + b + lo) == key) ? b + lo : -1;
}

// Membership filter in front of the hash lookup: bit (top FB bits of hash32(y)) is set for every key,
// so a clear bit proves y is not in L (most probes miss; a miss then costs one shared load).
template <int FB>
__device__ __forceinline__ uint32_t filter_may_hold(const uint32_t* filt, int32_t y) {
    const uint32_t h = hash32((uint32_t)y) >> (32 - FB);
    const uint32_t w = filt[h >> 5];
    return __funnelshift_r(w, w, h) & 1u;  // bit (h mod 32) of the word: the rotate takes h mod 32
}

// single-graph mode: one block reduction and one atomic per statistic at the end of the kernel;
// the signature hits go to acc[ACC_SIG_HITS] in both modes
__device__ __forceinline__ void flush_block(const Sink& sink, uint64_t tri, uint64_t k4, uint64_t paw, uint64_t hits,
                                            uint64_t* red) {
    tri = block_sum_u64(tri, red);
    k4 = block_sum_u64(k4, red);
    paw = block_sum_u64(paw, red);
    hits = block_sum_u64(hits, red);
    if (threadIdx.x == 0) {
        if (hits) atomicAdd((unsigned long long*)&sink.acc[ACC_SIG_HITS], (unsigned long long)hits);
        if (!sink.batch()) {
            if (tri) atomicAdd((unsigned long long*)&sink.acc[ACC_T], (unsigned long long)tri);
            if (k4) atomicAdd((unsigned long long*)&sink.acc[ACC_K4], (unsigned long long)k4);
            if (paw) atomicAdd((unsigned long long*)&sink.acc[ACC_PAWSUM], (unsigned long long)paw);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Warp-local mode.
// ---------------------------------------------------------------------------------------------
constexpr int kWarpThreads = 256;
constexpr int kWarpsPerBlock = kWarpThreads / 32;
constexpr int kWarpHashBits = 7;  // 128 slots for <= 32 keys: load <= 1/4, ~1.4 slot reads per miss
constexpr int kWarpFilterBits = 10;  // membership filter of 1024 bits: false positives <= 32 / 1024

template <bool BS>
__global__ void __launch_bounds__(kWarpThreads, 4) k_tri_warp(const int64_t* __restrict__ offp,
                                                           const int32_t* __restrict__ colsp,
                                                           const int32_t* __restrict__ deg,
                                                           const int32_t* __restrict__ q,
                                                           const unsigned long long* __restrict__ cnt,
                                                           bool reuse, uint32_t* __restrict__ te, Sink sink) {
    __shared__ int32_t sL[kWarpsPerBlock][32];
    __shared__ uint32_t sRow[kWarpsPerBlock][32];
    __shared__ int32_t sHk[kWarpsPerBlock][1 << kWarpHashBits];
    __shared__ uint8_t sHv[kWarpsPerBlock][1 << kWarpHashBits];
    __shared__ uint32_t sFilt[kWarpsPerBlock][(1 << kWarpFilterBits) / 32];
    __shared__ uint64_t red[32];
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t nq = (int64_t)cnt[0];
    uint64_t tri = 0, k4 = 0, paw = 0, hits = 0;
    FilterChoice fc;
    for (int64_t k = ((int64_t)blockIdx.x * kWarpsPerBlock + w); k < nq; k += (int64_t)gridDim.x * kWarpsPerBlock) {
        const int32_t u = q[k];
        const int64_t ub = offp[u];
        const int d = (int)(offp[u + 1] - ub);
        const int32_t x = (l < d) ? colsp[ub + l] : kInf;
        sL[w][l] = x;
        sRow[w][l] = 0;
#pragma unroll
        for (int hs = 0; hs < (1 << kWarpHashBits); hs += 32) sHk[w][l + hs] = kNoKey;
        sFilt[w][l] = 0;
        __syncwarp();
        if (l < d) {
            if (!BS) hash_put(sHk[w], sHv[w], kWarpHashBits, x, l);
            const uint32_t h = hash32((uint32_t)x) >> (32 - kWarpFilterBits);
            atomicOr(&sFilt[w][h >> 5], 1u << (h & 31));
        }
        __syncwarp();
        const int32_t last = sL[w][d - 1];
        auto lookup = [&](int32_t y) {
            return BS ? find_sorted(sL[w], d, y) : hash_get(sHk[w], sHv[w], kWarpHashBits, y);
        };
        // every row at once, lane i for row i (the lanes' dependent loads overlap).  A row that searches
        // (see row_searches, judged on the whole of N+(L[i])) looks its keys up in the whole list: a key
        // found there is an edge wherever it lies, so the search needs no narrower range.  A row that
        // probes needs its exact range [myb, mye): the elements of N+(L[i]) in [L[i+1], max L] (a
        // smaller element could be a member of L before L[i+1])
        int64_t myb = 0, mye = 0;
        bool mysearch = false;
        if (l < d - 1) {
            const int64_t b0 = offp[x], e0 = offp[x + 1];
            mysearch = row_searches(d - 1 - l, e0 - b0);
            if (mysearch) {
                myb = b0;
                mye = e0;
            } else {
                myb = b0 + lower_bound_i32(colsp + b0, e0 - b0, sL[w][l + 1]);
                mye = myb + lower_bound_i32(colsp + myb, e0 - myb, sL[w][d - 1] + 1);
            }
        }
        // the searching rows' (row, key) pairs are flattened over the lanes, so one round of binary
        // searches covers several short rows; pair t belongs to the last row whose first pair is at or
        // before t
        const uint32_t searching = __ballot_sync(kFull, mysearch);
        const int npairs = mysearch ? d - 1 - l : 0;
        int incl = npairs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (l >= o) incl += y;
        }
        const int excl = incl - npairs;
        const int total = __shfl_sync(kFull, incl, 31);
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + l;
            int o = 0;
#pragma unroll
            for (int sft = 16; sft >= 1; sft >>= 1) {
                const int e = __shfl_sync(kFull, excl, o + sft);
                if (e <= t) o += sft;
            }
            const int64_t rb = __shfl_sync(kFull, myb, o), re = __shfl_sync(kFull, mye, o);
            const int oe = __shfl_sync(kFull, excl, o);
            if (t < total) {
                const int j = o + 1 + (t - oe);
                const int64_t p = find_in_range(colsp, rb, (int)(re - rb), sL[w][j]);
                if (p >= 0) {
                    atomicAdd(&te[p], 1u);  // arc (L[o], L[j]): top edge of triangle (u, L[o], L[j])
                    atomicOr(&sRow[w][o], 1u << j);
                }
            }
        }
        // the other rows probe their ranges
        for (int i = 0; i < d - 1; ++i) {
            if ((searching >> i) & 1u) continue;
            const int64_t b = __shfl_sync(kFull, myb, i), e = __shfl_sync(kFull, mye, i);
            uint32_t row = 0;
            probe_filtered(colsp, b, e, fc.use(),
                           [&](int32_t y) { return filter_may_hold<kWarpFilterBits>(sFilt[w], y); },
                           [&](int32_t y, int64_t p) {  // y is in [next, last] already
                               const int j = lookup(y);
                               if (j >= 0) {
                                   atomicAdd(&te[p], 1u);  // arc (v, y): top edge of triangle (u, v, y)
                                   row |= 1u << j;
                               }
                           });
            row = __reduce_or_sync(kFull, row);
            fc.add(e - b, (uint32_t)__popc(row));  // each set bit is one hit
            if (l == i) sRow[w][i] = row;
        }
        __syncwarp();
        uint32_t col = 0;  // # rows with bit l
        for (int i = 0; i < d - 1; ++i) col += (sRow[w][i] >> l) & 1u;
        const uint32_t myrow = sRow[w][l];
        const uint32_t own = (l < d) ? (uint32_t)__popc(myrow) + col : 0u;
        if (own) atomicAdd(&te[ub + l], own);
        const uint64_t a_tri = (uint64_t)__popc(myrow);
        uint64_t a_k4 = 0;
        uint32_t bits = myrow;
        if (reuse) {
            while (bits) {  // the staged frontier of (u, L[j]) answers the extension
                const int j = __ffs(bits) - 1;
                bits &= bits - 1;
                a_k4 += (uint64_t)__popc(myrow & sRow[w][j]);
            }
            hits += a_tri;
        } else {
            while (bits) {  // recompute |N+(L[j]) n S_uv| from N+(L[j]) in global memory
                const int j = __ffs(bits) - 1;
                bits &= bits - 1;
                const int32_t wv = sL[w][j];
                for (int64_t p = offp[wv], pe = offp[wv + 1]; p < pe; ++p) {
                    const int32_t y = colsp[p];
                    if (y > last) break;
                    const int jj = lookup(y);
                    if (jj >= 0 && ((myrow >> jj) & 1u)) ++a_k4;
                }
            }
        }
        const uint64_t dx = (l < d) ? (uint64_t)deg[x] : 0;
        const uint64_t a_paw = (uint64_t)own * dx + a_tri * (uint64_t)deg[u];
        if (sink.batch()) {
            const uint64_t t1 = warp_sum(a_tri), t2 = warp_sum(a_k4), t3 = warp_sum(a_paw);
            if (l == 0) {
                sink_add(sink, u, G_T, t1);
                sink_add(sink, u, G_K4, t2);
                sink_add(sink, u, G_PAWSUM, t3);
            }
        } else {
            tri += a_tri;
            k4 += a_k4;
            paw += a_paw;
        }
        __syncwarp();
    }
    flush_block(sink, tri, k4, paw, hits, red);
}

// ---------------------------------------------------------------------------------------------
// CTA mode: rows of the anchor's out-neighbourhood bitmap in shared memory.
// ---------------------------------------------------------------------------------------------
template <int DMAX>
struct CtaSmem {
    static constexpr int W = DMAX / 32;             // words per row
    static constexpr int WS = W | 1;                // odd row stride: no bank conflicts
    static constexpr int HB = (DMAX <= 256) ? 10 : ((DMAX <= 512) ? 11 : 12);  // 4 * DMAX hash slots
    // filter: 64 bits per key (2, 4 and 8 KB); false positives at most d / 2^FB <= 1 / 64
    static constexpr int FB = HB + 4;
    // The 256 and 1024 modes resolve every row's exact probe range up front (one binary search per
    // thread per bound); the 512 mode does so only for direct-table anchors (in the filter's bytes,
    // below) and otherwise finds each row's range with the warp-wide search when the row is taken:
    // two more range arrays would cost it a resident block per SM.
    static constexpr bool PRE = DMAX <= 256 || DMAX >= 1024;
    int32_t L[DMAX];
    uint32_t own[DMAX];
    uint32_t R[DMAX * WS];
    // membership of y in L: a direct table indexed by y - L[0] when L's span fits (tab[y - L[0]] = index
    // + 1, 0 = absent; 3 * 2^HB entries), else a hash of 2^HB slots in the same bytes
    static constexpr int TAB = 3 << HB;
    union {
        struct {
            int32_t hk[1 << HB];
            uint16_t hv[1 << HB];
        } h;
        uint16_t tab[TAB];
    } m;
    // the filter (hash and binary-search anchors) or, for direct-table anchors of the 512 mode, every
    // row's probe range as offsets into N+(L[i]): lo in rel[i], hi in rel[DMAX + i] (the same 8 * DMAX
    // bytes)
    union {
        uint32_t filt[(1 << FB) / 32];
        int32_t rel[2 * DMAX];
    };
    static_assert((1 << FB) / 32 == 2 * DMAX, "the filter and the relative ranges share their bytes");
    // row i probes colsp[rb[i], re[i]): the elements of N+(L[i]) in [L[i+1], max L]
    int64_t rb[PRE ? DMAX : 1];
    int64_t re[PRE ? DMAX : 1];
    uint64_t red[32];
};


template <int DMAX, int THREADS, int MINB, bool BS>
__global__ void __launch_bounds__(THREADS, MINB) k_tri_cta(const int64_t* __restrict__ offp,
                                                     const int32_t* __restrict__ colsp,
                                                     const int32_t* __restrict__ deg,
                                                     const int32_t* __restrict__ q, int64_t n, int cls,
                                                     int wmax, int cmax, int bmax, bool reuse,
                                                     const unsigned long long* __restrict__ cnt,
                                                     unsigned long long* __restrict__ ticket,
                                                     uint32_t* __restrict__ te, Sink sink) {
    using S = CtaSmem<DMAX>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S& s = *reinterpret_cast<S*>(smem_raw);
    __shared__ int64_t s_item;
    constexpr int NW = THREADS / 32;
    const int w = threadIdx.x >> 5, l = lane_id();
    const int64_t nq = (int64_t)cnt[1];
    uint64_t tri = 0, k4 = 0, paw = 0, hits = 0;
    FilterChoice fc;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(ticket, 1ull);
        __syncthreads();
        const int64_t k = s_item;
        __syncthreads();
        if (k >= nq) break;
        const int32_t u = q[n - 1 - k];
        const int64_t ub = offp[u];
        const int d = (int)(offp[u + 1] - ub);
        if (tri_class(d, wmax, cmax, bmax) != cls) continue;
        const int W = (d + 31) >> 5;
        const int WS = W | 1;
        // the direct table where L's span fits (dense anchors: high ranks, close together), the hash else
        const int32_t L0 = colsp[ub];
        const uint32_t span = (uint32_t)(colsp[ub + d - 1] - L0) + 1u;
        const bool direct = !BS && span <= (uint32_t)S::TAB;
        for (int i = threadIdx.x; i < d; i += THREADS) {
            s.L[i] = colsp[ub + i];
            s.own[i] = 0;
        }
        for (int i = threadIdx.x; i < d * WS; i += THREADS) s.R[i] = 0;
        if (direct) {
            for (int i = threadIdx.x; i < (int)span; i += THREADS) s.m.tab[i] = 0;
        } else {
            for (int i = threadIdx.x; i < (1 << S::HB); i += THREADS) s.m.h.hk[i] = kNoKey;
            for (int i = threadIdx.x; i < (1 << S::FB) / 32; i += THREADS) s.filt[i] = 0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < d; i += THREADS) {
            if (direct) {
                s.m.tab[s.L[i] - L0] = (uint16_t)(i + 1);
            } else {
                if (!BS) hash_put(s.m.h.hk, s.m.h.hv, S::HB, s.L[i], i);
                const uint32_t h = hash32((uint32_t)s.L[i]) >> (32 - S::FB);
                atomicOr(&s.filt[h >> 5], 1u << (h & 31));
            }
            if (!S::PRE && direct && i < d - 1) {  // the same, as offsets into N+(L[i]) (rows are short)
                const int32_t v = s.L[i];
                const int64_t b = offp[v], e = offp[v + 1];
                const int32_t lo = (int32_t)lower_bound_i32(colsp + b, e - b, s.L[i + 1]);
                s.rel[i] = lo;
                s.rel[DMAX + i] = lo + (int32_t)lower_bound_i32(colsp + b + lo, e - b - lo, s.L[d - 1] + 1);
            }
            if (S::PRE && i < d - 1) {  // every row's probe range at once: dependent loads overlap across rows
                const int32_t v = s.L[i];
                const int64_t b = offp[v], e = offp[v + 1];
                const int64_t lo = b + lower_bound_i32(colsp + b, e - b, s.L[i + 1]);
                s.rb[i] = lo;
                s.re[i] = lo + lower_bound_i32(colsp + lo, e - lo, s.L[d - 1] + 1);  // elements <= max L
            }
        }
        __syncthreads();
        const int32_t last = s.L[d - 1];
        // index of y in L, or -1
        auto find = [&](int32_t y) {
            if (direct) {
                const uint32_t o = (uint32_t)(y - L0);
                return o < span ? (int)s.m.tab[o] - 1 : -1;
            }
            return BS ? find_sorted(s.L, d, y) : hash_get(s.m.h.hk, s.m.h.hv, S::HB, y);
        };
        auto lookup = [&](int32_t y) {
            if (!direct && !filter_may_hold<S::FB>(s.filt, y)) return -1;
            return find(y);
        };
        // rows: warp per row, ordered intersection of N+(L[i]) with L over the exact range of N+(L[i]) in
        // [L[i+1], max L] (no smaller element can be in L after L[i], no larger one at all)
        for (int i = w; i < d - 1; i += NW) {
            int64_t b = 0, e = 0;
            if (S::PRE) {
                b = s.rb[i];
                e = s.re[i];
            } else if (direct) {
                const int64_t o = offp[s.L[i]];
                b = o + s.rel[i];
                e = o + s.rel[DMAX + i];
            } else {
                const int32_t v = s.L[i];
                const int64_t e0 = offp[v + 1];
                b = warp_lower_bound(colsp, offp[v], e0, s.L[i + 1]);
                e = warp_lower_bound(colsp, b, e0, last + 1);
            }
            uint32_t* Ri = &s.R[i * WS];
            uint32_t hits = 0;
            if (row_searches(d - 1 - i, e - b)) {  // the keys after L[i] searched in the range
                const int len = (int)(e - b);
                for (int j = i + 1 + l; j < d; j += 32) {
                    const int64_t p = find_in_range(colsp, b, len, s.L[j]);
                    if (p >= 0) {
                        atomicAdd(&te[p], 1u);  // arc (L[i], L[j]): top edge of triangle (u, L[i], L[j])
                        atomicOr(&Ri[j >> 5], 1u << (j & 31));
                        atomicAdd(&s.own[j], 1u);
                        ++hits;
                    }
                }
                hits = warp_sum(hits);
            } else {
                // the filter is built and used only with the hash or the binary search
                probe_filtered(colsp, b, e, !direct && fc.use(),
                               [&](int32_t y) { return filter_may_hold<S::FB>(s.filt, y); },
                               [&](int32_t y, int64_t p) {
                                   const int j = find(y);
                                   if (j >= 0) {
                                       atomicAdd(&te[p], 1u);  // arc (L[i], y): top edge of triangle (u, L[i], y)
                                       atomicOr(&Ri[j >> 5], 1u << (j & 31));
                                       atomicAdd(&s.own[j], 1u);
                                       ++hits;
                                   }
                               });
                hits = warp_sum(hits);
                fc.add(e - b, hits);
            }
            if (l == 0 && hits) atomicAdd(&s.own[i], hits);
        }
        __syncthreads();
        // triangles and 4-cliques (the X_3 extension): the bitmap's (word, row) units are dealt to all the
        // block's threads.  Unit (x, i) counts the set bits j of word x of row i (the triangles (u, L[i],
        // L[j])) and adds |row_i n row_j| for each, over the words from x on (row j has no bit at or
        // below j), so the work is spread by the bits themselves and no lane searches for its bit.  A
        // warp's lanes take one word of consecutive rows: equal word spans, conflict-free row reads.
        uint64_t a_tri = 0, a_k4 = 0, a_paw = 0;
        const int rows = d - 1;  // row d - 1 is empty
        for (int t = threadIdx.x; t < rows * W; t += THREADS) {
            const int x = t / rows, i = t - x * rows;
            if ((x << 5) + 31 <= i) continue;  // row i has no bit at or below i
            const uint32_t* Ri = &s.R[i * WS];
            uint32_t bits = Ri[x];
            a_tri += (uint64_t)__popc(bits);
            while (bits) {
                const int j = (x << 5) + __ffs(bits) - 1;
                bits &= bits - 1;
                uint32_t cnt = 0;
                if (reuse) {  // the staged frontier of (u, L[j])
                    const uint32_t* Rj = &s.R[j * WS];
                    for (int y = x; y < W; ++y) cnt += __popc(Ri[y] & Rj[y]);
                } else {      // recompute from N+(L[j]) in global memory
                    const int32_t wv = s.L[j];
                    for (int64_t p = offp[wv], pe = offp[wv + 1]; p < pe; ++p) {
                        const int32_t y = colsp[p];
                        if (y > last) break;
                        const int jj = lookup(y);
                        if (jj >= 0 && ((Ri[jj >> 5] >> (jj & 31)) & 1u)) ++cnt;
                    }
                }
                a_k4 += cnt;
            }
        }
        for (int i = threadIdx.x; i < d; i += THREADS) {
            const uint32_t o = s.own[i];
            if (o) {
                atomicAdd(&te[ub + i], o);
                a_paw += (uint64_t)o * (uint64_t)deg[s.L[i]];
            }
        }
        // the anchor's own degree term: T_u * d_u
        a_paw += a_tri * (uint64_t)deg[u];
        if (reuse) hits += a_tri;
        __syncthreads();
        if (sink.batch()) {
            const uint64_t t1 = block_sum_u64(a_tri, s.red);
            const uint64_t t2 = block_sum_u64(a_k4, s.red);
            const uint64_t t3 = block_sum_u64(a_paw, s.red);
            if (threadIdx.x == 0) {
                sink_add(sink, u, G_T, t1);
                sink_add(sink, u, G_K4, t2);
                sink_add(sink, u, G_PAWSUM, t3);
            }
        } else {
            tri += a_tri;
            k4 += a_k4;
            paw += a_paw;
        }
    }
    flush_block(sink, tri, k4, paw, hits, s.red);
}

// ---------------------------------------------------------------------------------------------
// Global-staged mode (kCtaMax < d <= kBigMax): one 512-thread block per anchor, the d rows of d bits
// in the block's slice of a global scratch (row stride W = ceil(d / 32) words; at most 2 MiB, so it
// stays in L2).  A warp builds one row at a time in its shared buffer (membership of y in L by binary
// search of the sorted L in shared memory) and writes it out; after a block barrier the 4-clique
// extension reads the staged rows back, exactly as the CTA mode does from shared memory.
// ---------------------------------------------------------------------------------------------
constexpr int kBigThreads = 512;
constexpr int kBigWarps = kBigThreads / 32;
constexpr int kBigWords = kBigMax / 32;

struct BigSmem {
    int32_t L[kBigMax];
    uint32_t own[kBigMax];
    uint32_t row[kBigWarps][kBigWords];
    uint64_t red[32];
};

__global__ void __launch_bounds__(kBigThreads, 1) k_tri_big(const int64_t* __restrict__ offp,
                                                            const int32_t* __restrict__ colsp,
                                                            const int32_t* __restrict__ deg,
                                                            const int32_t* __restrict__ q_big,
                                                            const unsigned long long* __restrict__ cnt_big,
                                                            unsigned long long* __restrict__ ticket, bool reuse,
                                                            uint32_t* __restrict__ scratch,
                                                            uint32_t* __restrict__ te, Sink sink) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BigSmem& s = *reinterpret_cast<BigSmem*>(smem_raw);
    __shared__ int64_t s_item;
    const int w = threadIdx.x >> 5, l = lane_id();
    uint32_t* R = scratch + (size_t)blockIdx.x * kBigMax * kBigWords;
    uint32_t* buf = s.row[w];
    const int64_t nq = (int64_t)*cnt_big;
    uint64_t tri = 0, k4 = 0, paw = 0, hits = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(ticket, 1ull);
        __syncthreads();
        const int64_t k = s_item;
        __syncthreads();
        if (k >= nq) break;
        const int32_t u = q_big[k];
        const int64_t ub = offp[u];
        const int d = (int)(offp[u + 1] - ub);  // cmax < d <= kBigMax by classification
        const int W = (d + 31) >> 5;
        for (int i = threadIdx.x; i < d; i += kBigThreads) {
            s.L[i] = colsp[ub + i];
            s.own[i] = 0;
        }
        __syncthreads();
        const int32_t last = s.L[d - 1];
        // rows: warp per row, built in the warp's shared buffer, then written to the scratch
        for (int i = w; i < d; i += kBigWarps) {
            for (int x = l; x < W; x += 32) buf[x] = 0;
            __syncwarp();
            uint32_t hits_i = 0;
            if (i < d - 1) {
                const int32_t v = s.L[i];
                const int32_t next = s.L[i + 1];
                const int64_t e = offp[v + 1];
                int64_t b = offp[v];
                if (e - b > 64) b = warp_lower_bound(colsp, b, e, next);
                auto probe = [&](int32_t y, int64_t p) {
                    if (y >= next && y <= last) {
                        const int j = find_sorted(s.L, d, y);
                        if (j >= 0) {
                            atomicAdd(&te[p], 1u);
                            atomicOr(&buf[j >> 5], 1u << (j & 31));
                            atomicAdd(&s.own[j], 1u);
                            ++hits_i;
                        }
                    }
                };
                probe_list(colsp, b, e, last, probe);
            }
            hits_i = warp_sum(hits_i);
            if (l == 0 && hits_i) atomicAdd(&s.own[i], hits_i);
            __syncwarp();
            for (int x = l; x < W; x += 32) R[(size_t)i * W + x] = buf[x];
            __syncwarp();
        }
        __syncthreads();  // every row is in the scratch
        uint64_t a_tri = 0, a_k4 = 0, a_paw = 0;
        for (int i = w; i < d - 1; i += kBigWarps) {
            const uint32_t* Ri = R + (size_t)i * W;
            for (int x = l; x < W; x += 32) buf[x] = Ri[x];
            __syncwarp();
            // the set bits of row i in chunks of 32 words (one word per lane), dealt to the lanes
            for (int c0 = 0; c0 < W; c0 += 32) {
                const uint32_t myw = c0 + l < W ? buf[c0 + l] : 0u;
                const int cnt_w = __popc(myw);
                int pre = cnt_w;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, pre, o);
                    if (l >= o) pre += y;
                }
                const int B = __shfl_sync(kFull, pre, 31);
                pre -= cnt_w;
                a_tri += (l == 0) ? (uint64_t)B : 0;
                for (int k0 = 0; k0 < B; k0 += 32) {
                    const int kk = k0 + l;
                    int o = 0;
#pragma unroll
                    for (int sft = 16; sft >= 1; sft >>= 1) {
                        const int e = __shfl_sync(kFull, pre, o + sft);
                        if (e <= kk) o += sft;
                    }
                    const uint32_t word = __shfl_sync(kFull, myw, o);
                    const int rank = kk - __shfl_sync(kFull, pre, o);
                    if (kk < B) {
                        const int j = ((c0 + o) << 5) + (int)__fns(word, 0, rank + 1);
                        uint32_t cnt = 0;
                        if (reuse) {  // the staged frontier of (u, L[j])
                            const uint32_t* Rj = R + (size_t)j * W;
                            for (int x = c0 + o; x < W; ++x) cnt += __popc(buf[x] & Rj[x]);
                        } else {      // recompute from N+(L[j]) in global memory
                            const int32_t wv = s.L[j];
                            for (int64_t p = offp[wv], pe = offp[wv + 1]; p < pe; ++p) {
                                const int32_t y = colsp[p];
                                if (y > last) break;
                                const int jj = find_sorted(s.L, d, y);
                                if (jj >= 0 && ((buf[jj >> 5] >> (jj & 31)) & 1u)) ++cnt;
                            }
                        }
                        a_k4 += cnt;
                    }
                }
            }
            __syncwarp();
        }
        for (int i = threadIdx.x; i < d; i += kBigThreads) {
            const uint32_t o = s.own[i];
            if (o) {
                atomicAdd(&te[ub + i], o);
                a_paw += (uint64_t)o * (uint64_t)deg[s.L[i]];
            }
        }
        a_paw += a_tri * (uint64_t)deg[u];
        if (reuse) hits += a_tri;
        __syncthreads();
        if (sink.batch()) {
            const uint64_t t1 = block_sum_u64(a_tri, s.red);
            const uint64_t t2 = block_sum_u64(a_k4, s.red);
            const uint64_t t3 = block_sum_u64(a_paw, s.red);
            if (threadIdx.x == 0) {
                sink_add(sink, u, G_T, t1);
                sink_add(sink, u, G_K4, t2);
                sink_add(sink, u, G_PAWSUM, t3);
            }
        } else {
            tri += a_tri;
            k4 += a_k4;
            paw += a_paw;
        }
    }
    flush_block(sink, tri, k4, paw, hits, s.red);
}

// ---------------------------------------------------------------------------------------------
// Fallback for out-degree > kCtaMax (1024): per out-arc (u, v) the frontier S_uv = N+(u) n N+(v) is
// materialised (compaction) in a per-warp global buffer, then reused for the 4-clique extension.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t lb_global(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t y) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < y) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_tri_fallback(const int64_t* __restrict__ offp,
                                                      const int32_t* __restrict__ colsp,
                                                      const int32_t* __restrict__ deg,
                                                      const int32_t* __restrict__ q_fb,
                                                      const unsigned long long* __restrict__ cnt_fb,
                                                      int32_t* __restrict__ scratch, int64_t scratch_per_warp,
                                                      uint32_t* __restrict__ te, Sink sink) {
    __shared__ uint64_t red[32];
    const int w = threadIdx.x >> 5, l = lane_id();
    const int nw = blockDim.x >> 5;
    int32_t* S = scratch + ((int64_t)blockIdx.x * nw + w) * scratch_per_warp;
    const int64_t nq = (int64_t)*cnt_fb;
    uint64_t tri = 0, k4 = 0, paw = 0;
    for (int64_t k = blockIdx.x; k < nq; k += gridDim.x) {
        const int32_t u = q_fb[k];
        const int64_t ub = offp[u], ue = offp[u + 1];
        const uint64_t du = (uint64_t)deg[u];
        const uint64_t tri0 = tri, k40 = k4, paw0 = paw;
        for (int64_t a = ub + w; a < ue; a += nw) {  // warp per out-arc (u, v)
            const int32_t v = colsp[a];
            const int64_t b = offp[v], e = offp[v + 1];
            const uint64_t dv = (uint64_t)deg[v];
            int64_t ns = 0;
            uint32_t own_uv = 0;
            for (int64_t p0 = b; p0 < e; p0 += 32) {
                const int64_t p = p0 + l;
                bool hit = false;
                int32_t y = kInf;
                int64_t pu = 0;
                if (p < e) {
                    y = colsp[p];
                    pu = lb_global(colsp, ub, ue, y);
                    hit = pu < ue && colsp[pu] == y;
                }
                const uint32_t hm = __ballot_sync(kFull, hit);
                if (hit) {
                    atomicAdd(&te[p], 1u);   // (v, y)
                    atomicAdd(&te[pu], 1u);  // (u, y)
                    S[ns + __popc(hm & lanemask_lt())] = y;
                    paw += du + dv + (uint64_t)deg[y];
                }
                ns += __popc(hm);
                own_uv += __popc(hm);
            }
            if (l == 0 && own_uv) atomicAdd(&te[a], own_uv);
            tri += (l == 0) ? (uint64_t)own_uv : 0;
            __syncwarp();
            // 4-cliques through (u, v): pairs w < x of S_uv with x in N+(w)
            for (int64_t s1 = 0; s1 < ns; ++s1) {
                const int32_t wv = S[s1];
                const int64_t wb = offp[wv], we = offp[wv + 1];
                for (int64_t s2 = s1 + 1 + l; s2 < ns; s2 += 32) {
                    const int32_t xv = S[s2];
                    const int64_t px = lb_global(colsp, wb, we, xv);
                    k4 += (px < we && colsp[px] == xv) ? 1 : 0;
                }
            }
            __syncwarp();
        }
        if (sink.batch()) {  // this anchor's part goes to its graph; the running sums stay unchanged
            const uint64_t t1 = block_sum_u64(tri - tri0, red);
            const uint64_t t2 = block_sum_u64(k4 - k40, red);
            const uint64_t t3 = block_sum_u64(paw - paw0, red);
            if (threadIdx.x == 0) {
                sink_add(sink, u, G_T, t1);
                sink_add(sink, u, G_K4, t2);
                sink_add(sink, u, G_PAWSUM, t3);
            }
            tri = tri0;
            k4 = k40;
            paw = paw0;
        }
    }
    flush_block(sink, tri, k4, paw, 0, red);
}

template <int DMAX, int THREADS, int MINB, bool BS>
harp_status launch_cta(const harp_csr* g, Workspace& ws, int cls, int ticket_slot, int wmax, int cmax, int bmax,
                       bool reuse, cudaStream_t s) {
    const size_t smem = sizeof(CtaSmem<DMAX>);
    HARP_CK(cudaFuncSetAttribute(k_tri_cta<DMAX, THREADS, MINB, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    k_tri_cta<DMAX, THREADS, MINB, BS><<<num_sms() * MINB, THREADS, smem, s>>>(
        ws.offp, ws.colsp, ws.deg, ws.q_tri, g->n, cls, wmax, cmax, bmax, reuse,
        (const unsigned long long*)&ws.acc[Q_TRI_WARP], (unsigned long long*)&ws.acc[ticket_slot], ws.te,
        Sink{ws.acc, ws.gid, ws.accG});
    HARP_LAUNCHED();
    return HARP_OK;
}

// The four staged tiers, each with its bin's membership probe (plan.tri_probe_bin[k]: bsearch or hash).
harp_status launch_tiers(const harp_csr* g, Workspace& ws, int wmax, int cmax, int bmax, bool reuse,
                         const uint8_t* probe_bin, cudaStream_t s) {
    const Sink sink{ws.acc, ws.gid, ws.accG};
    const bool bs0 = probe_bin[0] == HARP_PROBE_BSEARCH, bs1 = probe_bin[1] == HARP_PROBE_BSEARCH;
    const bool bs2 = probe_bin[2] == HARP_PROBE_BSEARCH, bs3 = probe_bin[3] == HARP_PROBE_BSEARCH;
    const unsigned wgrid = (unsigned)num_sms() * 8;
    const unsigned long long* qcnt = (const unsigned long long*)&ws.acc[Q_TRI_WARP];
    if (bs0) k_tri_warp<true><<<wgrid, kWarpThreads, 0, s>>>(ws.offp, ws.colsp, ws.deg, ws.q_tri, qcnt, reuse, ws.te, sink);
    else k_tri_warp<false><<<wgrid, kWarpThreads, 0, s>>>(ws.offp, ws.colsp, ws.deg, ws.q_tri, qcnt, reuse, ws.te, sink);
    HARP_LAUNCHED();
    HARP_CK(prof_mark(s, SEG_TRI_WARP));
    if (bs1) HARP_TRY((launch_cta<kCta1, kCta1Threads, kCta1Blocks, true>(g, ws, 1, T_TRI_S, wmax, cmax, bmax, reuse, s)));
    else HARP_TRY((launch_cta<kCta1, kCta1Threads, kCta1Blocks, false>(g, ws, 1, T_TRI_S, wmax, cmax, bmax, reuse, s)));
    HARP_CK(prof_mark(s, SEG_TRI_CTA_S));
    if (bs2) HARP_TRY((launch_cta<kCta2, 256, 4, true>(g, ws, 2, T_TRI_M, wmax, cmax, bmax, reuse, s)));
    else HARP_TRY((launch_cta<kCta2, 256, 4, false>(g, ws, 2, T_TRI_M, wmax, cmax, bmax, reuse, s)));
    if (bs3) HARP_TRY((launch_cta<kCtaMax, 1024, 1, true>(g, ws, 3, T_TRI_L, wmax, cmax, bmax, reuse, s)));
    else HARP_TRY((launch_cta<kCtaMax, 1024, 1, false>(g, ws, 3, T_TRI_L, wmax, cmax, bmax, reuse, s)));
    HARP_CK(prof_mark(s, SEG_TRI_CTA_L));
    return HARP_OK;
}

}  // namespace

// acc[Q_TRI_WARP], acc[Q_TRI_CTA] hold the queue lengths, acc[T_TRI_*] the CTA tickets (all cleared
// with the accumulators before the count).
harp_status count_triangles_k4(const harp_csr* g, Workspace& ws, const harp_plan& plan, cudaStream_t s) {
    const int64_t n = g->n;
    if (n == 0 || g->m == 0) return HARP_OK;  // no marks: the segments read as zero
    const int wmax = (int)plan.tri_warp_max;  // normalised: 1..32
    const int cmax = (int)plan.tri_cta_max;   // normalised: 1..kCtaMax
    const int bmax = (int)plan.tri_big_max;   // normalised: 1..kBigMax
    const bool reuse = !(plan.flags & HARP_PLAN_NO_REUSE);
    unsigned long long* cnt = (unsigned long long*)&ws.acc[Q_TRI_WARP];
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    unsigned long long* cnt_fb = (unsigned long long*)&ws.acc[Q_TRI_FB];
    unsigned long long* cnt_big = (unsigned long long*)&ws.acc[Q_TRI_BIG];
    k_tri_classify<<<(unsigned)blocks, 256, 0, s>>>(ws.dplus, n, ws.own_lo, ws.own_hi, wmax, cmax, bmax, ws.q_tri,
                                                    ws.q_mid, cnt, cnt_fb, cnt_big);
    HARP_LAUNCHED();
    const Sink sink{ws.acc, ws.gid, ws.accG};
    HARP_TRY(launch_tiers(g, ws, wmax, cmax, bmax, reuse, plan.tri_probe_bin, s));
    // the largest possible out-degree is bounded by sqrt(2m) and by the maximum degree
    int64_t dmax = 1;
    while (dmax * dmax < 2 * g->m) ++dmax;
    if (dmax > g->max_deg) dmax = g->max_deg;
    if (dmax > cmax && bmax > cmax) {  // global-staged tier: one block per SM, scratch of kBigMax rows
        const size_t bytes = (size_t)num_sms() * kBigMax * kBigWords * sizeof(uint32_t);
        uint32_t* scratch = nullptr;
        HARP_CK(cudaMallocAsync((void**)&scratch, bytes, s));
        const size_t smem = sizeof(BigSmem);
        cudaError_t e = cudaFuncSetAttribute(k_tri_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            k_tri_big<<<num_sms(), kBigThreads, smem, s>>>(ws.offp, ws.colsp, ws.deg, ws.q_mid + n, cnt_big,
                                                      (unsigned long long*)&ws.acc[T_TRI_BIG], reuse, scratch, ws.te,
                                                      sink);
            note_launch();
            e = cudaGetLastError();
        }
        cudaFreeAsync(scratch, s);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            return HARP_ECUDA;
        }
    }
    // fallback: per-warp frontier buffers of the largest possible out-degree
    if (dmax > cmax && dmax > bmax) {
        const int fb_blocks = num_sms();
        const int64_t per_warp = dmax + 32;
        const size_t bytes = (size_t)fb_blocks * 8 * (size_t)per_warp * sizeof(int32_t);
        int32_t* scratch = nullptr;
        HARP_CK(cudaMallocAsync((void**)&scratch, bytes, s));
        k_tri_fallback<<<fb_blocks, 256, 0, s>>>(ws.offp, ws.colsp, ws.deg, ws.q_mid, cnt_fb, scratch, per_warp,
                                                 ws.te, sink);
        note_launch();
        cudaError_t e = cudaGetLastError();
        cudaFreeAsync(scratch, s);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            return HARP_ECUDA;
        }
    }
    HARP_CK(prof_mark(s, SEG_TRI_FALLBACK));
    return HARP_OK;
}

}  // namespace harp
