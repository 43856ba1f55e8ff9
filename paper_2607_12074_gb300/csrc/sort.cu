// Device-wide LSD radix sort of 64-bit keys (8-bit digits, stable per pass).
//
// Per pass: (1) every 2048-key tile counts its digits; (2) one exclusive scan over the
// digit-major histogram gives each (digit, tile) its output base; (3) every tile ranks its keys
// stably with __match_any_sync peer groups inside each warp and a per-warp running count per digit,
// then scatters.  Tiles, warps within a tile, rounds within a warp and lanes within a round are
// ordered as the input, which makes every pass stable.
#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // 2048
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kRsThreads) k_radix_upsweep(const uint64_t* __restrict__ keys, int64_t n,
                                                              int shift, uint32_t mask,
                                                              uint32_t* __restrict__ hist, int64_t nb) {
    __shared__ uint32_t cnt[kRadix];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        int64_t i = base + k * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRsThreads) k_radix_downsweep(const uint64_t* __restrict__ keys,
                                                                uint64_t* __restrict__ out, int64_t n,
                                                                int shift, uint32_t mask,
                                                                const uint32_t* __restrict__ hist,
                                                                int64_t nb) {
    __shared__ uint32_t wcnt[kRsWarps][kRadix];
    __shared__ uint32_t gbase[kRadix];
    const int w = threadIdx.x >> 5, l = lane_id();
    for (int d = threadIdx.x; d < kRsWarps * kRadix; d += kRsThreads) (&wcnt[0][0])[d] = 0;
    gbase[threadIdx.x] = hist[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * (kRsItems * 32);
    uint64_t key[kRsItems];
    uint32_t dig[kRsItems];
    uint32_t rank[kRsItems];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        int64_t i = base + k * 32 + l;
        bool valid = i < n;
        key[k] = valid ? keys[i] : 0;
        uint32_t d = valid ? ((uint32_t)(key[k] >> shift) & mask) : (uint32_t)kRadix;
        dig[k] = d;
        uint32_t peers = __match_any_sync(kFull, d);
        uint32_t r = __popc(peers & lt);
        uint32_t prior = valid ? wcnt[w][d] : 0;
        __syncwarp();
        if (valid && r == 0) wcnt[w][d] += __popc(peers);
        __syncwarp();
        rank[k] = prior + r;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // one digit per thread (kRsThreads == kRadix)
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ++ww) {
            uint32_t c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        if (dig[k] < (uint32_t)kRadix) {
            uint32_t pos = gbase[dig[k]] + wcnt[w][dig[k]] + rank[k];
            out[pos] = key[k];
        }
    }
}

}  // namespace

size_t radix_hist_len(int64_t n) {
    int64_t nb = (n + kRsTile - 1) / kRsTile;
    if (nb < 1) nb = 1;
    return (size_t)nb * kRadix + 1;
}

harp_status radix_sort_u64(uint64_t** keys, uint64_t** alt, int64_t n, int begin_bit, int end_bit,
                           uint32_t* hist, int64_t* tmp, size_t tmp_len, cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return HARP_OK;
    if (n > (int64_t)0xFFFFFFFFLL) return HARP_EOVERFLOW;  // positions are 32-bit
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        const int bits = (end_bit - shift) < 8 ? (end_bit - shift) : 8;
        const uint32_t mask = (1u << bits) - 1u;
        k_radix_upsweep<<<(unsigned)nb, kRsThreads, 0, s>>>(*keys, n, shift, mask, hist, nb);
        HARP_LAUNCHED();
        HARP_TRY(exclusive_scan_u32_inplace(hist, nb * kRadix, tmp, tmp_len, s));
        k_radix_downsweep<<<(unsigned)nb, kRsThreads, 0, s>>>(*keys, *alt, n, shift, mask, hist, nb);
        HARP_LAUNCHED();
        uint64_t* t = *keys;
        *keys = *alt;
        *alt = t;
    }
    return HARP_OK;
}

}  // namespace harp
