// Step a1: degree ordering and orientation (Section III-D, "sorted CSR adjacency and canonical
// ordering constraints").
//
// Vertices are renumbered by rank(v) = (d(v), v) ascending, so that in the new numbering
//   * N+(v) = neighbours ranked above v = the suffix of v's sorted row after v itself,
//   * N-(v) = neighbours ranked below v = the prefix of the row,
//   * the neighbours of w ranked below u form a prefix of w's row (the ordered wedges of the
//     4-cycle anchor, Section III-B, read contiguous memory).
// Output (workspace): deg, order (new -> old), perm (old -> new), off/cols (relabelled CSR with
// every row sorted), dplus, offp/colsp (out-CSR: only N+), te zeroed, S = sum_v C(d_v, 3).
//
// Rows are sorted by four kernels chosen by degree: for d <= 32 a lane's bitonic network in registers
// (d <= 16) or the warp's over its lanes (every row is visited), a warp bitonic sort in the warp's
// shared buffer for d <= 256, a block bitonic sort in shared memory for d <= 4096 and a per-row LSD
// radix sort through global memory for hubs (the last three from queues filled by the relabel pass;
// the warp and block sorts share one).
#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kTierA = 32;
constexpr int kTierB1 = 256;
constexpr int kTierB = 4096;

int bits_for(int64_t x) {
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) <= x) ++b;
    return b < 1 ? 1 : b;
}

unsigned grid_for(int64_t work, int threads, int64_t cap = -1) {
    if (cap < 0) cap = (int64_t)num_sms() * 64;
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

__global__ void k_vertex_keys(const int64_t* __restrict__ off, int64_t n, int b, int bd,
                              uint64_t* __restrict__ keys, uint64_t* __restrict__ acc,
                              const int32_t* __restrict__ gid_in, uint64_t* __restrict__ accG) {
    uint64_t s3 = 0;
    // a caller-built CSR that failed its check (harp_count4_noalloc) is counted as edgeless: every
    // later kernel then stays inside the arrays sized for its (n, m)
    const bool bad_csr = (acc[ACC_ERR] & kErrBadCsr) != 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d = bad_csr ? 0 : (uint64_t)(off[v + 1] - off[v]);
        const uint64_t g = gid_in ? (uint64_t)gid_in[v] : 0;
        keys[v] = (g << (bd + b)) | (d << b) | (uint64_t)v;
        const uint64_t c3 = choose3_u64(d);
        if (gid_in) {
            if (c3) atomicAdd((unsigned long long*)&accG[(int64_t)gid_in[v] * kGStride + G_S], (unsigned long long)c3);
        } else {
            s3 += c3;
        }
    }
    __shared__ uint64_t red[32];
    uint64_t t = block_sum_u64(s3, red);
    if (threadIdx.x == 0 && t) atomicAdd((unsigned long long*)&acc[ACC_S], (unsigned long long)t);
}

// New ids = sorted key order.  Rows that need the CTA or hub sort are queued (q: CTA rows from the
// front, hub rows from the back); the warp sort takes every other row directly.
__global__ void k_relabel(const uint64_t* __restrict__ keys, int64_t n, int b, int bd, int32_t* __restrict__ order,
                          int32_t* __restrict__ perm, int32_t* __restrict__ deg,
                          const int32_t* __restrict__ gid_in, int32_t* __restrict__ gid,
                          int32_t* __restrict__ q, unsigned long long* __restrict__ qcnt) {
    const uint64_t mask = ((uint64_t)1 << b) - 1;
    const uint64_t dmask = ((uint64_t)1 << bd) - 1;
    const int l = lane_id();
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - l; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + l;
        int cls = -1;
        if (i < n) {
            const uint64_t k = keys[i];
            const int32_t old = (int32_t)(k & mask);
            const int32_t d = (int32_t)((k >> b) & dmask);
            order[i] = old;
            perm[old] = (int32_t)i;
            deg[i] = d;
            if (gid_in) gid[i] = gid_in[old];
            cls = d > kTierB ? 1 : (d > kTierA ? 0 : -1);
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint32_t m = __ballot_sync(kFull, cls == c);
            if (!m) continue;
            unsigned long long start = 0;
            const int leader = __ffs(m) - 1;
            if (l == leader) start = atomicAdd(&qcnt[c], (unsigned long long)__popc(m));
            start = __shfl_sync(kFull, start, leader);
            if (cls == c) {
                const unsigned long long k = start + __popc(m & lanemask_lt());
                if (c == 0) q[k] = (int32_t)i;
                else q[n - 1 - (int64_t)k] = (int32_t)i;
            }
        }
    }
}

// Tier A: rows with 1 <= d <= 32, 32 consecutive rows per warp (consecutive ranks have similar
// degrees).  A row of at most 16 neighbours is sorted by its own lane, a bitonic network over 8 or 16
// registers padded with +inf; the warp then sorts its rows of 17..32 together, a bitonic network over
// the lanes.  A warp per row left most lanes idle on the many short rows of sparse graphs.
template <int P>
__device__ __forceinline__ void sort_regs(int32_t (&a)[P]) {
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int p = i ^ j;
                if (p > i) {
                    const int32_t lo = min(a[i], a[p]), hi = max(a[i], a[p]);
                    const bool up = (i & k) == 0;
                    a[i] = up ? lo : hi;
                    a[p] = up ? hi : lo;
                }
            }
        }
    }
}

template <int P>
__device__ __forceinline__ void lane_sort_row(int64_t i, int d, const int64_t* __restrict__ goff,
                                              const int32_t* __restrict__ gcols, const int32_t* __restrict__ order,
                                              const int32_t* __restrict__ perm, const int64_t* __restrict__ off,
                                              int32_t* __restrict__ cols, int32_t* __restrict__ dplus) {
    const int64_t src = goff[order[i]];
    int32_t a[P];
#pragma unroll
    for (int r = 0; r < P; ++r) a[r] = r < d ? perm[gcols[src + r]] : 0x7fffffff;
    sort_regs<P>(a);
    const int64_t ob = off[i];
    int above = 0;
#pragma unroll
    for (int r = 0; r < P; ++r) {
        if (r < d) {
            cols[ob + r] = a[r];
            above += a[r] > (int32_t)i;
        }
    }
    dplus[i] = above;
}

__global__ void __launch_bounds__(256) k_sort_rows_warp(const int64_t* __restrict__ goff,
                                                        const int32_t* __restrict__ gcols,
                                                        const int32_t* __restrict__ order,
                                                        const int32_t* __restrict__ perm,
                                                        const int32_t* __restrict__ deg,
                                                        const int64_t* __restrict__ off, int64_t n,
                                                        int32_t* __restrict__ cols,
                                                        int32_t* __restrict__ dplus) {
    const int l = lane_id();
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i0 = wid * 32; i0 < n; i0 += nw * 32) {
        const int64_t i = i0 + l;
        const int d = i < n ? deg[i] : -1;  // CTA and hub rows (d > 32) are sorted by the queued kernels
        if (d == 0) dplus[i] = 0;
        else if (d >= 1 && d <= 8) lane_sort_row<8>(i, d, goff, gcols, order, perm, off, cols, dplus);
        else if (d > 8 && d <= 16) lane_sort_row<16>(i, d, goff, gcols, order, perm, off, cols, dplus);
        uint32_t rest = __ballot_sync(kFull, d > 16 && d <= kTierA);
        while (rest) {
            const int src = __ffs(rest) - 1;
            rest &= rest - 1;
            const int64_t r = i0 + src;
            const int dr = __shfl_sync(kFull, d, src);
            const int64_t rsrc = goff[order[r]];
            int32_t v = (l < dr) ? perm[gcols[rsrc + l]] : 0x7fffffff;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    int32_t o = __shfl_xor_sync(kFull, v, j);
                    bool up = (l & k) == 0;
                    bool lower = (l & j) == 0;
                    v = (lower == up) ? min(v, o) : max(v, o);
                }
            }
            if (l < dr) cols[off[r] + l] = v;
            uint32_t above = __ballot_sync(kFull, l < dr && v > (int32_t)r);
            if (l == 0) dplus[r] = __popc(above);
        }
    }
}

// Tier B1: 32 < d <= 256, one warp per row, bitonic sort in the warp's shared buffer (a block per
// row would leave most of its warps idle behind a block barrier at every stage).
constexpr int kMidWarps = 8;

__global__ void __launch_bounds__(kMidWarps * 32) k_sort_rows_mid(const int64_t* __restrict__ goff,
                                                                   const int32_t* __restrict__ gcols,
                                                                   const int32_t* __restrict__ order,
                                                                   const int32_t* __restrict__ perm,
                                                                   const int32_t* __restrict__ deg,
                                                                   const int64_t* __restrict__ off, int64_t n,
                                                                   int32_t* __restrict__ cols,
                                                                   int32_t* __restrict__ dplus,
                                                                   const int32_t* __restrict__ q,
                                                                   const unsigned long long* __restrict__ qcnt) {
    __shared__ int32_t sbuf[kMidWarps][kTierB1];
    const int w = threadIdx.x >> 5, l = lane_id();
    int32_t* buf = sbuf[w];
    const int64_t nq = (int64_t)qcnt[0];
    for (int64_t qi = (int64_t)blockIdx.x * kMidWarps + w; qi < nq; qi += (int64_t)gridDim.x * kMidWarps) {
        const int64_t i = q[qi];
        const int d = deg[i];
        if (d > kTierB1) continue;  // the block sort's row
        int P = 64;
        while (P < d) P <<= 1;
        const int64_t src = goff[order[i]];
        for (int k = l; k < P; k += 32) buf[k] = (k < d) ? perm[gcols[src + k]] : 0x7fffffff;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = l; t < (P >> 1); t += 32) {
                    const int a = 2 * t - (t & (j - 1));  // index with bit j clear
                    const int c = a + j;
                    const bool up = (a & k) == 0;
                    const int32_t x = buf[a], y = buf[c];
                    if ((x > y) == up) {
                        buf[a] = y;
                        buf[c] = x;
                    }
                }
                __syncwarp();
            }
        }
        int below = 0;
        for (int k = l; k < d; k += 32) {
            const int32_t x = buf[k];
            cols[off[i] + k] = x;
            below += x < (int32_t)i;
        }
        below = warp_sum(below);
        if (l == 0) dplus[i] = d - below;
        __syncwarp();  // every lane has read the buffer before the next row fills it
    }
}

// Tier B: 256 < d <= 4096, one block per row, bitonic sort in shared memory.
__global__ void __launch_bounds__(512) k_sort_rows_block(const int64_t* __restrict__ goff,
                                                         const int32_t* __restrict__ gcols,
                                                         const int32_t* __restrict__ order,
                                                         const int32_t* __restrict__ perm,
                                                         const int32_t* __restrict__ deg,
                                                         const int64_t* __restrict__ off, int64_t n,
                                                         int32_t* __restrict__ cols,
                                                         int32_t* __restrict__ dplus,
                                                         const int32_t* __restrict__ q,
                                                         const unsigned long long* __restrict__ qcnt) {
    __shared__ int32_t buf[kTierB];
    __shared__ int cnt_below;
    const int64_t nq = (int64_t)qcnt[0];
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int64_t i = q[qi];
        const int d = deg[i];
        if (d <= kTierB1) continue;  // the warp sort's row (the same value in every thread)
        int P = 64;
        while (P < d) P <<= 1;
        const int64_t src = goff[order[i]];
        for (int k = threadIdx.x; k < P; k += blockDim.x) buf[k] = (k < d) ? perm[gcols[src + k]] : 0x7fffffff;
        if (threadIdx.x == 0) cnt_below = 0;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                    int a = 2 * t - (t & (j - 1));  // index with bit j clear
                    int c = a + j;
                    bool up = (a & k) == 0;
                    int32_t x = buf[a], y = buf[c];
                    if ((x > y) == up) {
                        buf[a] = y;
                        buf[c] = x;
                    }
                }
                __syncthreads();
            }
        }
        int below = 0;
        for (int k = threadIdx.x; k < d; k += blockDim.x) {
            int32_t x = buf[k];
            cols[off[i] + k] = x;
            below += x < (int32_t)i;
        }
        below = warp_sum(below);
        if (lane_id() == 0 && below) atomicAdd(&cnt_below, below);
        __syncthreads();
        if (threadIdx.x == 0) dplus[i] = d - cnt_below;
        __syncthreads();
    }
}

// Tier C: hubs (d > 4096), one block per row, LSD radix sort (8-bit digits) through global memory.
// Pass p reads the previous pass's output; pass 0 reads the old row through perm.  The pass count
// decides which buffer each pass writes so that the last one lands in `cols`.
constexpr int kHubThreads = 512;
constexpr int kHubWarps = kHubThreads / 32;

__global__ void __launch_bounds__(kHubThreads) k_sort_rows_hub(const int64_t* __restrict__ goff,
                                                               const int32_t* __restrict__ gcols,
                                                               const int32_t* __restrict__ order,
                                                               const int32_t* __restrict__ perm,
                                                               const int32_t* __restrict__ deg,
                                                               const int64_t* __restrict__ off, int64_t n,
                                                               int nbits, int32_t* __restrict__ cols,
                                                               int32_t* __restrict__ tmp,
                                                               int32_t* __restrict__ dplus,
                                                               const int32_t* __restrict__ q,
                                                               const unsigned long long* __restrict__ qcnt) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[kHubWarps][256];
    __shared__ int cnt_below;
    const int npass = (nbits + 7) / 8;
    const int w = threadIdx.x >> 5, l = lane_id();
    const uint32_t lt = lanemask_lt();
    const int64_t nq = (int64_t)qcnt[1];
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int64_t i = q[n - 1 - qi];
        const int64_t d = deg[i];
        const int64_t src = goff[order[i]];
        const int64_t dst0 = off[i];
        for (int p = 0; p < npass; ++p) {
            const int shift = 8 * p;
            const bool to_cols = ((npass - 1 - p) & 1) == 0;
            int32_t* out = (to_cols ? cols : tmp) + dst0;
            const int32_t* in = (p == 0) ? nullptr : ((to_cols ? tmp : cols) + dst0);
            // histogram of the row
            for (int k = threadIdx.x; k < 256; k += blockDim.x) base[k] = 0;
            __syncthreads();
            for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
                int32_t x = in ? in[k] : perm[gcols[src + k]];
                atomicAdd(&base[((uint32_t)x >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x < 32) {  // exclusive scan of 256 counters by one warp
                uint32_t c[8], s = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) { c[q] = base[threadIdx.x * 8 + q]; s += c[q]; }
                uint32_t inc = s;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t u = __shfl_up_sync(kFull, inc, o);
                    if (threadIdx.x >= o) inc += u;
                }
                uint32_t run = inc - s;
#pragma unroll
                for (int q = 0; q < 8; ++q) { base[threadIdx.x * 8 + q] = run; run += c[q]; }
            }
            __syncthreads();
            // stable scatter, tile by tile (tile = kHubThreads keys, warp-contiguous)
            for (int64_t t0 = 0; t0 < d; t0 += kHubThreads) {
                for (int k = threadIdx.x; k < kHubWarps * 256; k += blockDim.x) (&wcnt[0][0])[k] = 0;
                __syncthreads();
                const int64_t k = t0 + w * 32 + l;
                const bool valid = k < d;
                int32_t x = 0;
                if (valid) x = in ? in[k] : perm[gcols[src + k]];
                const uint32_t dg = valid ? (((uint32_t)x >> shift) & 255u) : 256u;
                const uint32_t peers = __match_any_sync(kFull, dg);
                const uint32_t r = __popc(peers & lt);
                if (valid && r == 0) wcnt[w][dg] = __popc(peers);
                __syncthreads();
                if (threadIdx.x < 256) {  // exclusive over warps, add the running digit base
                    uint32_t run = base[threadIdx.x];
                    for (int ww = 0; ww < kHubWarps; ++ww) {
                        uint32_t c = wcnt[ww][threadIdx.x];
                        wcnt[ww][threadIdx.x] = run;
                        run += c;
                    }
                    base[threadIdx.x] = run;
                }
                __syncthreads();
                if (valid) out[wcnt[w][dg] + r] = x;
                __syncthreads();
            }
            __syncthreads();
        }
        // out-degree: elements above i in the sorted row
        if (threadIdx.x == 0) cnt_below = 0;
        __syncthreads();
        int below = 0;
        for (int64_t k = threadIdx.x; k < d; k += blockDim.x) below += cols[dst0 + k] < (int32_t)i;
        below = warp_sum(below);
        if (l == 0 && below) atomicAdd(&cnt_below, below);
        __syncthreads();
        if (threadIdx.x == 0) dplus[i] = (int32_t)(d - cnt_below);
        __syncthreads();
    }
}

// colsp[offp[i] + k] = the k-th neighbour of i ranked above i (the row suffix), 32 consecutive rows
// per warp: a lane copies its own row when the suffix has at most 32 entries, the warp copies the
// longer ones together.  The same pass accumulates sum over edges of (d_u - 1)(d_v - 1) (3-edge paths
// + 3T).
__global__ void __launch_bounds__(256) k_out_csr(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                                 const int32_t* __restrict__ dplus,
                                                 const int32_t* __restrict__ deg,
                                                 const int64_t* __restrict__ offp, int64_t n,
                                                 int32_t* __restrict__ colsp, Sink sink) {
    __shared__ uint64_t red[32];
    const int l = lane_id();
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t pw = 0;
    for (int64_t i0 = wid * 32; i0 < n; i0 += nw * 32) {
        const int64_t i = i0 + l;
        const int64_t dp = i < n ? dplus[i] : 0;
        if (dp > 0 && dp <= 32) {
            const int64_t srcb = off[i + 1] - dp;
            const int64_t dstb = offp[i];
            const uint64_t di1 = (uint64_t)deg[i] - 1;
            uint64_t row_pw = 0;
            for (int64_t k = 0; k < dp; ++k) {
                const int32_t v = cols[srcb + k];
                colsp[dstb + k] = v;
                row_pw += di1 * ((uint64_t)deg[v] - 1);
            }
            if (sink.batch()) sink_add(sink, (int32_t)i, G_PW, row_pw);
            else pw += row_pw;
        }
        uint32_t rest = __ballot_sync(kFull, dp > 32);
        while (rest) {
            const int src = __ffs(rest) - 1;
            rest &= rest - 1;
            const int64_t r = i0 + src;
            const int64_t rdp = __shfl_sync(kFull, dp, src);
            const int64_t srcb = off[r + 1] - rdp;
            const int64_t dstb = offp[r];
            const uint64_t di1 = (uint64_t)deg[r] - 1;
            uint64_t row_pw = 0;
            for (int64_t k = l; k < rdp; k += 32) {
                const int32_t v = cols[srcb + k];
                colsp[dstb + k] = v;
                row_pw += di1 * ((uint64_t)deg[v] - 1);
            }
            if (sink.batch()) {
                row_pw = warp_sum(row_pw);
                if (l == 0) sink_add(sink, (int32_t)r, G_PW, row_pw);
            } else {
                pw += row_pw;
            }
        }
    }
    pw = block_sum_u64(pw, red);
    if (threadIdx.x == 0 && pw) atomicAdd((unsigned long long*)&sink.acc[ACC_PW], (unsigned long long)pw);
}

}  // namespace

harp_status orient(const harp_csr* g, Workspace& ws, cudaStream_t s) {
    const int64_t n = g->n, m = g->m;
    if (n == 0) return HARP_OK;
    const int b = bits_for(n);
    const int bd = bits_for(g->max_deg);
    const int bg = ws.gid_in && ws.G > 1 ? bits_for(ws.G - 1) : 0;
    if (b + bd + bg > 64) return HARP_EOVERFLOW;

    // rank = (graph, degree, id): each graph's vertices form one contiguous rank range, sorted by
    // degree (a single graph is graph 0)
    k_vertex_keys<<<grid_for(n, 256), 256, 0, s>>>(g->off, n, b, bd, ws.vkeys, ws.acc, ws.gid_in, ws.accG);
    HARP_LAUNCHED();
    uint64_t* k0 = ws.vkeys;
    uint64_t* k1 = ws.vkeys_alt;
    // the keys are written in id order and every pass is stable, so only the graph and degree bits
    // need sorting: equal (graph, degree) keep ascending ids
    HARP_TRY(radix_sort_u64(&k0, &k1, n, b, b + bd + bg, ws.hist, ws.scan_tmp, ws.scan_tmp_len, s));
    unsigned long long* qsort = (unsigned long long*)&ws.acc[Q_SORT_CTA];
    k_relabel<<<grid_for(n, 256), 256, 0, s>>>(k0, n, b, bd, ws.order, ws.perm, ws.deg, ws.gid_in, ws.gid, ws.q_tri,
                                               qsort);
    HARP_LAUNCHED();
    HARP_TRY(exclusive_scan_i32_to_i64(ws.deg, ws.off, n, ws.scan_tmp, ws.scan_tmp_len, s));
    if (m > 0) {
        // 32 rows per warp
        k_sort_rows_warp<<<grid_for(n, 256), 256, 0, s>>>(g->off, g->cols, ws.order, ws.perm, ws.deg,
                                                                ws.off, n, ws.cols, ws.dplus);
        HARP_LAUNCHED();
        k_sort_rows_mid<<<num_sms() * 8, kMidWarps * 32, 0, s>>>(g->off, g->cols, ws.order, ws.perm, ws.deg,
                                                                 ws.off, n, ws.cols, ws.dplus, ws.q_tri, qsort);
        HARP_LAUNCHED();
        k_sort_rows_block<<<num_sms() * 4, 512, 0, s>>>(g->off, g->cols, ws.order, ws.perm, ws.deg, ws.off, n,
                                                   ws.cols, ws.dplus, ws.q_tri, qsort);
        HARP_LAUNCHED();
        // the out-CSR columns + t_e region (2m int32) is free until k_out_csr: hub sort ping-pong
        k_sort_rows_hub<<<num_sms(), kHubThreads, 0, s>>>(g->off, g->cols, ws.order, ws.perm, ws.deg, ws.off, n, b,
                                                     ws.cols, ws.colsp, ws.dplus, ws.q_tri, qsort);
        HARP_LAUNCHED();
    } else {
        HARP_CK(cudaMemsetAsync(ws.dplus, 0, (size_t)n * sizeof(int32_t), s));
    }
    HARP_TRY(exclusive_scan_i32_to_i64(ws.dplus, ws.offp, n, ws.scan_tmp, ws.scan_tmp_len, s));
    if (m > 0) {
        const Sink sink{ws.acc, ws.gid, ws.accG};
        // 32 rows per warp
        k_out_csr<<<grid_for(n, 256), 256, 0, s>>>(ws.off, ws.cols, ws.dplus, ws.deg, ws.offp, n, ws.colsp,
                                                         sink);
        HARP_LAUNCHED();
        HARP_CK(cudaMemsetAsync(ws.te, 0, (size_t)m * sizeof(uint32_t), s));
    }
    return HARP_OK;
}

}  // namespace harp
