// Device-wide exclusive prefix sums (tile reduce -> scan of tile sums -> tile scan).
#include "harp_internal.cuh"

namespace harp {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(kFull, v, o);
        if (lane_id() >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; *total receives the block sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
    const int w = threadIdx.x >> 5, l = lane_id();
    T inc = warp_inclusive_scan(v);
    if (l == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T x = (l < (kScanThreads >> 5)) ? warp_tot[l] : T(0);
        T xi = warp_inclusive_scan(x);
        if (l < (kScanThreads >> 5)) warp_tot[l] = xi - x;
        if (l == (kScanThreads >> 5) - 1) *total = xi;
    }
    __syncthreads();
    T r = warp_tot[w] + inc - v;
    __syncthreads();
    return r;
}

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_tile_reduce(const Tin* __restrict__ in, int64_t n,
                                                              int64_t* __restrict__ partial) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) s += (int64_t)in[i];
    }
    __shared__ uint64_t red[32];
    uint64_t t = block_sum_u64((uint64_t)s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = (int64_t)t;
}

// out[i] = prefix(i) + partial[block];  out[n] = grand total (written by the last block).
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const Tin* in, Tout* out, int64_t n,
                                                            const int64_t* __restrict__ partial) {
    __shared__ int64_t tile[kScanTile];
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = (i < n) ? (int64_t)in[i] : 0;
    }
    __syncthreads();
    int64_t loc[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = tile[threadIdx.x * kScanItems + k];
        sum += loc[k];
    }
    int64_t pre = block_exclusive_scan<int64_t>(sum, warp_tot, &tot);
    const int64_t off = partial ? partial[blockIdx.x] : 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        tile[threadIdx.x * kScanItems + k] = pre + off;
        pre += loc[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = (Tout)tile[k * kScanThreads + threadIdx.x];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (Tout)(off + tot);
}

int64_t ntiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// In-place exclusive scan of an int64 array of length n (n + 1 entries written; data must have
// room for n + 1).  tmp holds the deeper levels.
harp_status scan_i64_inplace(int64_t* data, int64_t n, int64_t* tmp, size_t tmp_len, cudaStream_t s) {
    const int64_t nb = ntiles(n);
    if (nb <= 1) {
        k_tile_scan<int64_t, int64_t><<<1, kScanThreads, 0, s>>>(data, data, n, nullptr);
        HARP_LAUNCHED();
        return HARP_OK;
    }
    if ((size_t)(nb + 1) > tmp_len) return HARP_ENOMEM;
    k_tile_reduce<int64_t><<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, tmp);
    HARP_LAUNCHED();
    HARP_TRY(scan_i64_inplace(tmp, nb, tmp + nb + 1, tmp_len - (size_t)(nb + 1), s));
    k_tile_scan<int64_t, int64_t><<<(unsigned)nb, kScanThreads, 0, s>>>(data, data, n, tmp);
    HARP_LAUNCHED();
    return HARP_OK;
}

}  // namespace

size_t scan_tmp_needed(int64_t n) {
    size_t need = 0;
    int64_t x = n;
    while (true) {
        int64_t nb = ntiles(x);
        if (nb <= 1) break;
        need += (size_t)nb + 1;
        x = nb;
    }
    return need + 64;
}

harp_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* tmp,
                                      size_t tmp_len, cudaStream_t s) {
    const int64_t nb = ntiles(n);
    if (nb <= 1) {
        k_tile_scan<int32_t, int64_t><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        HARP_LAUNCHED();
        return HARP_OK;
    }
    if ((size_t)(nb + 1) > tmp_len) return HARP_ENOMEM;
    k_tile_reduce<int32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    HARP_LAUNCHED();
    HARP_TRY(scan_i64_inplace(tmp, nb, tmp + nb + 1, tmp_len - (size_t)(nb + 1), s));
    k_tile_scan<int32_t, int64_t><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
    HARP_LAUNCHED();
    return HARP_OK;
}

harp_status exclusive_scan_u32_inplace(uint32_t* data, int64_t n, int64_t* tmp, size_t tmp_len,
                                       cudaStream_t s) {
    // In-place form over n entries: entry i receives sum_{j<i} data[j]; the last input value is
    // not needed for that, so the tile scan runs over n - 1 values and writes its total at n - 1.
    if (n <= 0) return HARP_OK;
    const int64_t nb = ntiles(n);
    if (nb <= 1) {
        // single tile; write the total into a scratch slot instead of data[n]
        if (tmp_len < 2) return HARP_ENOMEM;
        k_tile_scan<uint32_t, uint32_t><<<1, kScanThreads, 0, s>>>(data, data, n - 1, nullptr);
        HARP_LAUNCHED();
        return HARP_OK;
    }
    if ((size_t)(nb + 1) > tmp_len) return HARP_ENOMEM;
    k_tile_reduce<uint32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, tmp);
    HARP_LAUNCHED();
    HARP_TRY(scan_i64_inplace(tmp, nb, tmp + nb + 1, tmp_len - (size_t)(nb + 1), s));
    k_tile_scan<uint32_t, uint32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(data, data, n - 1, tmp);
    HARP_LAUNCHED();
    return HARP_OK;
}

}  // namespace harp
