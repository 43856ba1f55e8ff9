// Step a7: the last anchor statistic (sum_e C(t_e, 2)) and the closure (Section III-F).
//
// The closure equations of Section III-F, written per anchor in the paper
//   N_paw = sum_T X_1(T),  N_diamond = 1/2 sum_T X_2(T),  N_clique4 = 1/4 sum_T X_3(T),
//   N_path4 / N_cycle4 from the A_e x B_e pairs of every edge,
//   N_star = sum_u [C(d,3) - m(H_u)(d-2) + sum_{v in N(u)} C(deg_H v, 2) - tau(H_u)],
// are the same linear system as the containment of non-induced patterns in induced classes:
//   S   = star + paw + 2 diamond + 4 K4            (S   = sum_v C(d_v, 3))
//   P   = path + 2 paw + 4 C4 + 6 diamond + 12 K4  (P   = sum_e (d_u-1)(d_v-1) - 3T)
//   paw'= paw + 4 diamond + 12 K4                  (paw'= sum over triangles of (d_a+d_b+d_c-6))
//   C4' = C4 + diamond + 3 K4                      (C4' = wedge-anchor 4-cycles)
//   D   = diamond + 6 K4                           (D   = sum_e C(t_e, 2))
// (e.g. sum_v m(H_v)(d_v-2) = paw', sum_v sum_{w in N(v)} C(deg_H w, 2) = 2D, sum_v tau(H_v) = 4 K4 turn
// the star equation into star = S - paw' + 2D - 4K4).  The system is unit upper-triangular in the
// order K4, diamond, C4, paw, path, star, so back-substitution needs no division and is exact modulo
// 2^64: every count is exact whenever its true value is below 2^64.
#include "harp_internal.cuh"

namespace harp {
namespace {

__global__ void __launch_bounds__(256) k_reduce_close(const uint32_t* __restrict__ te, int64_t m,
                                                      uint64_t* __restrict__ acc) {
    __shared__ uint64_t red[32];
    __shared__ bool last;
    uint64_t dsum = 0;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x)
        dsum += choose2_u64((uint64_t)te[a]);
    dsum = block_sum_u64(dsum, red);
    if (threadIdx.x == 0) {
        if (dsum) atomicAdd((unsigned long long*)&acc[ACC_D], (unsigned long long)dsum);
        __threadfence();
        const unsigned long long done = atomicAdd((unsigned long long*)&acc[ACC_DONE], 1ull);
        last = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    volatile uint64_t* va = acc;
    const uint64_t T = va[ACC_T], K4 = va[ACC_K4], C4n = va[ACC_C4], S = va[ACC_S];
    const uint64_t P = va[ACC_PW] - 3 * T;
    const uint64_t pawn = va[ACC_PAWSUM] - 6 * T;
    const uint64_t D = va[ACC_D];
    const uint64_t diamond = D - 6 * K4;
    const uint64_t c4 = C4n - diamond - 3 * K4;
    const uint64_t paw = pawn - 4 * diamond - 12 * K4;
    const uint64_t path = P - 2 * paw - 4 * c4 - 6 * diamond - 12 * K4;
    const uint64_t star = S - paw - 2 * diamond - 4 * K4;
    acc[OUT_COUNTS + HARP_STAR3] = star;
    acc[OUT_COUNTS + HARP_PATH4] = path;
    acc[OUT_COUNTS + HARP_PAW] = paw;
    acc[OUT_COUNTS + HARP_CYCLE4] = c4;
    acc[OUT_COUNTS + HARP_DIAMOND] = diamond;
    acc[OUT_COUNTS + HARP_CLIQUE4] = K4;
    acc[OUT_STATS + HARP_STAT_TRIANGLES] = T;
    acc[OUT_STATS + HARP_STAT_K4] = K4;
    acc[OUT_STATS + HARP_STAT_C4] = C4n;
    acc[OUT_STATS + HARP_STAT_STARS] = S;
    acc[OUT_STATS + HARP_STAT_PATHS] = P;
    acc[OUT_STATS + HARP_STAT_PAWS] = pawn;
    acc[OUT_STATS + HARP_STAT_DIAMONDS] = D;
    acc[OUT_STATS + HARP_STAT_EDGES] = (uint64_t)m;
}

// Batch mode: sum_e C(t_e, 2) per graph over the out-CSR rows, 32 consecutive rows per warp.  A lane
// sums its own row when it has at most 32 out-arcs, the warp sums the longer rows together; then one
// atomic per graph present among the warp's rows (ranks are ordered by graph first, so consecutive
// rows almost always share one) instead of one per row.
__global__ void __launch_bounds__(256) k_reduce_rows_batch(const int64_t* __restrict__ offp,
                                                           const uint32_t* __restrict__ te, int64_t n, Sink sink) {
    const int l = lane_id();
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u0 = wid * 32; u0 < n; u0 += nw * 32) {
        const int64_t u = u0 + l;
        int64_t b = 0, e = 0;
        int32_t g = -1;
        uint64_t d = 0;
        if (u < n) {
            b = offp[u];
            e = offp[u + 1];
            g = sink.gid[u];
            if (e - b <= 32)
                for (int64_t a = b; a < e; ++a) d += choose2_u64((uint64_t)te[a]);
        }
        uint32_t big = __ballot_sync(kFull, e - b > 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t rb = __shfl_sync(kFull, b, src), re = __shfl_sync(kFull, e, src);
            uint64_t rd = 0;
            for (int64_t a = rb + l; a < re; a += 32) rd += choose2_u64((uint64_t)te[a]);
            rd = warp_sum(rd);
            if (l == src) d = rd;
        }
        uint32_t left = __ballot_sync(kFull, d != 0);
        while (left) {  // one graph per round: the first lane still holding a sum names it
            const int src = __ffs(left) - 1;
            const int32_t gs = __shfl_sync(kFull, g, src);
            const bool mine = ((left >> l) & 1u) && g == gs;
            const uint64_t sum = warp_sum(mine ? d : (uint64_t)0);
            if (l == src)
                atomicAdd((unsigned long long*)&sink.accG[(int64_t)gs * kGStride + G_D], (unsigned long long)sum);
            left &= ~__ballot_sync(kFull, mine);
        }
    }
}

// Batch mode: the closure of every graph (one thread per graph); out holds 16 uint64 per graph.
__global__ void k_close_batch(const uint64_t* __restrict__ accG, int64_t G, uint64_t* __restrict__ out) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t* a = accG + g * kGStride;
        const uint64_t T = a[G_T], K4 = a[G_K4], C4n = a[G_C4], S = a[G_S];
        const uint64_t P = a[G_PW] - 3 * T;
        const uint64_t pawn = a[G_PAWSUM] - 6 * T;
        const uint64_t D = a[G_D];
        const uint64_t diamond = D - 6 * K4;
        const uint64_t c4 = C4n - diamond - 3 * K4;
        const uint64_t paw = pawn - 4 * diamond - 12 * K4;
        const uint64_t path = P - 2 * paw - 4 * c4 - 6 * diamond - 12 * K4;
        const uint64_t star = S - paw - 2 * diamond - 4 * K4;
        uint64_t* o = out + g * 16;
        o[HARP_STAR3] = star;
        o[HARP_PATH4] = path;
        o[HARP_PAW] = paw;
        o[HARP_CYCLE4] = c4;
        o[HARP_DIAMOND] = diamond;
        o[HARP_CLIQUE4] = K4;
        o[6] = 0;
        o[7] = 0;
        o[8 + HARP_STAT_TRIANGLES] = T;
        o[8 + HARP_STAT_K4] = K4;
        o[8 + HARP_STAT_C4] = C4n;
        o[8 + HARP_STAT_STARS] = S;
        o[8 + HARP_STAT_PATHS] = P;
        o[8 + HARP_STAT_PAWS] = pawn;
        o[8 + HARP_STAT_DIAMONDS] = D;
        o[8 + HARP_STAT_EDGES] = 0;  // filled by the host, which knows every member's m
    }
}

}  // namespace

harp_status reduce_and_close_batch(const harp_csr* g, Workspace& ws, int64_t G, uint64_t* d_out, cudaStream_t s) {
    const Sink sink{ws.acc, ws.gid, ws.accG};
    int64_t blocks = (g->n + 255) / 256;  // a lane per row
    if (blocks < 1) blocks = 1;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (g->m > 0) {
        k_reduce_rows_batch<<<(unsigned)blocks, 256, 0, s>>>(ws.offp, ws.te, g->n, sink);
        HARP_LAUNCHED();
    }
    int64_t cb = (G + 255) / 256;
    if (cb < 1) cb = 1;
    k_close_batch<<<(unsigned)cb, 256, 0, s>>>(ws.accG, G, d_out);
    HARP_LAUNCHED();
    return HARP_OK;
}

harp_status reduce_and_close(const harp_csr* g, Workspace& ws, cudaStream_t s) {
    int64_t blocks = (g->m + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    k_reduce_close<<<(unsigned)blocks, 256, 0, s>>>(ws.te, g->m, ws.acc);
    HARP_LAUNCHED();
    return HARP_OK;
}

}  // namespace harp
