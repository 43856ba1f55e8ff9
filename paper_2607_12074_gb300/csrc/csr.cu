// harp_build_csr on the device: canonical arc keys -> radix sort -> dedupe -> CSR.
//
// Every input pair (u, v), u != v, yields the arcs u->v and v->u as 64-bit keys (u << b) | v with
// b = bits(n).  Self-loops and out-of-range ids become a sentinel that sorts last (out-of-range ids
// also raise a flag that turns into HARP_EINVAL).  After the sort, the first copy of every key is
// kept; row offsets are the positions where the source id changes.
#include "harp_internal.cuh"

namespace harp {
namespace {

__global__ void k_make_arc_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                int64_t m_in, int64_t n, int b, uint64_t sentinel,
                                uint64_t* __restrict__ keys, unsigned int* __restrict__ bad) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m_in;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = src[e], v = dst[e];
        bool ok = u >= 0 && v >= 0 && (int64_t)u < n && (int64_t)v < n;
        if (!ok) atomicOr(bad, 1u);
        if (!ok || u == v) {
            keys[2 * e] = sentinel;
            keys[2 * e + 1] = sentinel;
        } else {
            keys[2 * e] = ((uint64_t)u << b) | (uint64_t)v;
            keys[2 * e + 1] = ((uint64_t)v << b) | (uint64_t)u;
        }
    }
}

__global__ void k_unique_flags(const uint64_t* __restrict__ keys, int64_t len, uint64_t sentinel,
                               int32_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        flag[i] = (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
}

__global__ void k_compact_cols(const uint64_t* __restrict__ keys, const int32_t* __restrict__ flag,
                               const int64_t* __restrict__ pos, int64_t len, uint64_t low_mask,
                               int32_t* __restrict__ cols, uint64_t* __restrict__ ckeys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            int64_t p = pos[i];
            cols[p] = (int32_t)(keys[i] & low_mask);
            ckeys[p] = keys[i];
        }
    }
}

// off[x] = first position whose source id is >= x (positions of the compacted, sorted arcs).
__global__ void k_row_offsets(const uint64_t* __restrict__ ckeys, int64_t M, int64_t n, int b,
                              int64_t* __restrict__ off) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = (int64_t)(ckeys[p] >> b);
        int64_t up = p > 0 ? (int64_t)(ckeys[p - 1] >> b) : -1;
        for (int64_t x = up + 1; x <= u; ++x) off[x] = p;
        if (p == M - 1)
            for (int64_t x = u + 1; x <= n; ++x) off[x] = M;
    }
}

__global__ void k_fill_i64(int64_t* __restrict__ a, int64_t len, int64_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_max_degree(const int64_t* __restrict__ off, int64_t n, unsigned long long* __restrict__ out) {
    int64_t best = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = off[v + 1] - off[v];
        best = d > best ? d : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t other = __shfl_xor_sync(kFull, best, o);
        best = other > best ? other : best;
    }
    if (lane_id() == 0) atomicMax(out, (unsigned long long)best);
}

unsigned grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (int64_t)num_sms() * 32) b = (int64_t)num_sms() * 32;
    return (unsigned)b;
}

int bits_for(int64_t x) {  // number of bits to represent x (x >= 0)
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) <= x) ++b;
    return b < 1 ? 1 : b;
}

}  // namespace

harp_status build_csr_device(harp_csr* g, int64_t n, int64_t m_in, const int32_t* d_src,
                             const int32_t* d_dst, cudaStream_t s) {
    const int b = bits_for(n);
    const uint64_t sentinel = ((uint64_t)n << b) | (uint64_t)n;
    const int64_t len = 2 * m_in;
    harp_status st = HARP_OK;

    uint64_t *keys = nullptr, *alt = nullptr;
    int32_t* flag = nullptr;
    int64_t* pos = nullptr;
    uint32_t* hist = nullptr;
    int64_t* tmp = nullptr;
    unsigned long long* small = nullptr;  // [0] bad flag, [1] max degree
    const size_t tmp_len = scan_tmp_needed(len > 0 ? len : 1) + scan_tmp_needed((int64_t)radix_hist_len(len));
    const size_t hist_len = radix_hist_len(len);

    auto cleanup = [&]() {
        if (keys) cudaFreeAsync(keys, s);
        if (alt) cudaFreeAsync(alt, s);
        if (flag) cudaFreeAsync(flag, s);
        if (pos) cudaFreeAsync(pos, s);
        if (hist) cudaFreeAsync(hist, s);
        if (tmp) cudaFreeAsync(tmp, s);
        if (small) cudaFreeAsync(small, s);
    };
#define BCK(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) {                               \
            record_cuda_error(e_);                             \
            cleanup();                                         \
            return e_ == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA; \
        }                                                      \
    } while (0)
#define BTRY(call)                                             \
    do {                                                       \
        st = (call);                                           \
        if (st != HARP_OK) { cleanup(); return st; }           \
    } while (0)

    BCK(cudaMallocAsync((void**)&small, 2 * sizeof(unsigned long long), s));
    BCK(cudaMemsetAsync(small, 0, 2 * sizeof(unsigned long long), s));
    BCK(cudaMallocAsync((void**)&g->off, (size_t)(n + 1) * sizeof(int64_t), s));
    int64_t M = 0;
    if (len > 0) {
        BCK(cudaMallocAsync((void**)&keys, (size_t)len * sizeof(uint64_t), s));
        BCK(cudaMallocAsync((void**)&alt, (size_t)len * sizeof(uint64_t), s));
        BCK(cudaMallocAsync((void**)&flag, (size_t)len * sizeof(int32_t), s));
        BCK(cudaMallocAsync((void**)&pos, (size_t)(len + 1) * sizeof(int64_t), s));
        BCK(cudaMallocAsync((void**)&hist, hist_len * sizeof(uint32_t), s));
        BCK(cudaMallocAsync((void**)&tmp, tmp_len * sizeof(int64_t), s));
        k_make_arc_keys<<<grid_for(m_in, 256), 256, 0, s>>>(d_src, d_dst, m_in, n, b, sentinel, keys,
                                                             (unsigned int*)small);
        note_launch();
        BCK(cudaGetLastError());
        BTRY(radix_sort_u64(&keys, &alt, len, 0, 2 * b, hist, tmp, tmp_len, s));
        k_unique_flags<<<grid_for(len, 256), 256, 0, s>>>(keys, len, sentinel, flag);
        note_launch();
        BCK(cudaGetLastError());
        BTRY(exclusive_scan_i32_to_i64(flag, pos, len, tmp, tmp_len, s));
        BCK(cudaMemcpyAsync(&M, pos + len, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    }
    unsigned long long bad = 0;
    BCK(cudaMemcpyAsync(&bad, small, sizeof(bad), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (bad) {
        cleanup();
        return HARP_EINVAL;
    }
    g->n = n;
    g->m = M / 2;
    BCK(cudaMallocAsync((void**)&g->cols, (size_t)(M > 0 ? M : 1) * sizeof(int32_t), s));
    g->csr_bytes = (size_t)(n + 1) * sizeof(int64_t) + (size_t)(M > 0 ? M : 1) * sizeof(int32_t);
    if (M > 0) {
        // reuse `alt` for the compacted keys
        k_compact_cols<<<grid_for(len, 256), 256, 0, s>>>(keys, flag, pos, len, ((uint64_t)1 << b) - 1,
                                                           g->cols, alt);
        note_launch();
        BCK(cudaGetLastError());
        k_row_offsets<<<grid_for(M, 256), 256, 0, s>>>(alt, M, n, b, g->off);
        note_launch();
        BCK(cudaGetLastError());
        k_max_degree<<<grid_for(n, 256), 256, 0, s>>>(g->off, n, small + 1);
        note_launch();
        BCK(cudaGetLastError());
    } else {
        k_fill_i64<<<grid_for(n + 1, 256), 256, 0, s>>>(g->off, n + 1, 0);
        note_launch();
        BCK(cudaGetLastError());
    }
    unsigned long long md = 0;
    BCK(cudaMemcpyAsync(&md, small + 1, sizeof(md), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    g->max_deg = (int64_t)md;
    cleanup();
    return HARP_OK;
#undef BCK
#undef BTRY
}

}  // namespace harp
