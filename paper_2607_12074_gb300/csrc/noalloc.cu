// harp_count4_noalloc: the counting pipeline for small graphs with every scratch buffer carved out
// of one file-scope static device array, so the call allocates nothing.
//
// Who needs it: callers that must not allocate device memory while they run - code executing
// inside another framework's pre-reserved memory regime, long-running services that forbid
// cudaMalloc/cudaFree after start-up (allocation can synchronise the device and fragment a
// carefully sized pool), and host threads that only own a stream.  They pass a device-resident CSR
// and a device output buffer; the library uses the static array below for everything else.
//
// The array lives in every process that loads libharp, on every GPU the process uses, until exit.
// All calls share it: two calls whose work overlaps on a GPU (different streams, or different host
// threads) race on it and give undefined results; serialise them (same stream, or events).
#include <mutex>

#include "harp_internal.cuh"

namespace harp {
namespace {

// Size limits of the static scratch.  m <= 2^19 also keeps every out-degree <= 1024 (out-degree is
// at most sqrt(2m)), so no execution mode that would need extra scratch is reached.
constexpr int64_t kNoAllocMaxN = 262144;
constexpr int64_t kNoAllocMaxM = 524288;
constexpr size_t kNoAllocBytes = (size_t)64 << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};  // device address of g_noalloc_scratch, per device

// The caller's CSR must match the sizes it passes: off[0] = 0, off[n] = 2m, offsets non-decreasing
// with every degree at most n - 1, and every column id in [0, n).  The offsets are checked first;
// the columns are read only when the offsets passed (so no read goes past off[n] = 2m).  A failure
// sets kErrBadCsr in acc[ACC_ERR]; the orientation pass then treats the graph as edgeless, so no
// kernel indexes past the scratch laid out for (n, m).
__global__ void k_check_offsets(const int64_t* __restrict__ off, int64_t n, int64_t m, uint64_t* __restrict__ acc) {
    bool bad = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = off[v];
        if (v == 0 && o != 0) bad = true;
        if (v == n && o != 2 * m) bad = true;
        if (v < n) {
            const int64_t d = off[v + 1] - o;
            if (d < 0 || d > n - 1) bad = true;
        }
    }
    if (__any_sync(kFull, bad) && lane_id() == 0) atomicOr((unsigned long long*)&acc[ACC_ERR], (unsigned long long)kErrBadCsr);
}

__global__ void k_check_cols(const int32_t* __restrict__ cols, int64_t n, int64_t m, uint64_t* __restrict__ acc) {
    // offsets failed: off[n] may not bound the columns.  Lane 0 reads the flag for its warp, so the
    // warp leaves (or stays) as a whole even while other warps set the same bit.
    const uint64_t flag = __shfl_sync(kFull, lane_id() == 0 ? acc[ACC_ERR] : 0ull, 0);
    if (flag & kErrBadCsr) return;
    bool bad = false;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < 2 * m; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cols[a];
        if (c < 0 || (int64_t)c >= n) bad = true;
    }
    if (__any_sync(kFull, bad) && lane_id() == 0) atomicOr((unsigned long long*)&acc[ACC_ERR], (unsigned long long)kErrBadCsr);
}

unsigned check_grid(int64_t work) {
    int64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)(b > cap ? cap : b);
}

// Lay out a Workspace for (n, m) inside [base, base + cap) with the library's one layout; returns
// the bytes used, or 0 if it does not fit.
size_t carve(unsigned char* base, size_t cap, int64_t n, int64_t m, Workspace& ws) {
    Workspace probe;
    const size_t need = ws_layout(probe, nullptr, n, m);
    if (need > cap) return 0;
    return ws_layout(ws, base, n, m);
}

// Device address of the static array for the current device (looked up once per device and kept
// for the life of the process: a device reset invalidates it, so the entry point must not be used
// across cudaDeviceReset).
harp_status scratch_address(unsigned char** out) {
    int dev = 0;
    HARP_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return HARP_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            record_cuda_error(e);
            return HARP_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    return HARP_OK;
}

}  // namespace
}  // namespace harp

using namespace harp;

extern "C" harp_status harp_count4_noalloc(int64_t n, int64_t m, const int64_t* d_offsets, const int32_t* d_cols,
                                           uint64_t* d_out, void* stream) {
    if (n < 0 || m < 0) return HARP_EINVAL;
    if (n > kNoAllocMaxN || m > kNoAllocMaxM) return HARP_ENOMEM;  // beyond the static scratch
    if (!d_out || (n > 0 && !d_offsets) || (m > 0 && !d_cols)) return HARP_EINVAL;
    unsigned char* base = nullptr;
    HARP_TRY(scratch_address(&base));
    harp_csr g;  // a view of the caller's CSR; owns nothing
    HARP_CK(cudaGetDevice(&g.device));
    cudaStream_t s = (cudaStream_t)stream;
    g.stream = s;
    g.n = n;
    g.m = m;
    g.max_deg = n > 0 ? n - 1 : 0;  // an upper bound suffices (it only sizes the degree sort key)
    g.off = const_cast<int64_t*>(d_offsets);
    g.cols = const_cast<int32_t*>(d_cols);
    Workspace ws;
    if (carve(base, kNoAllocBytes, n, m, ws) == 0) return HARP_ENOMEM;
    harp_plan plan;
    normalise_plan(nullptr, &plan);
    // every accumulator, queue counter and ticket starts at zero; the kernels clear t_e and the
    // window counts themselves
    HARP_CK(cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s));
    k_check_offsets<<<check_grid(n + 1), 256, 0, s>>>(d_offsets, n, m, ws.acc);
    HARP_LAUNCHED();
    if (m > 0) {
        k_check_cols<<<check_grid(2 * m), 256, 0, s>>>(d_cols, n, m, ws.acc);
        HARP_LAUNCHED();
    }
    if (n > 0) {
        HARP_TRY(orient(&g, ws, s));
        HARP_TRY(count_triangles_k4(&g, ws, plan, s));
        HARP_TRY(count_wedge_c4(&g, ws, plan, s));
    }
    HARP_TRY(reduce_and_close(&g, ws, s));
    HARP_CK(cudaMemcpyAsync(d_out, ws.acc, 16 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    HARP_CK(cudaMemcpyAsync(d_out + OUT_ERR, ws.acc + ACC_ERR, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return HARP_OK;
}
