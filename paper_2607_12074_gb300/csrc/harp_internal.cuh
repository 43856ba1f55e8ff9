// Internal declarations shared by the libharp translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "harp.h"

// ---------------------------------------------------------------------------------------------
// Error plumbing: every CUDA call is checked; the first failure is recorded per thread and the
// public entry point returns HARP_ECUDA.  No exceptions are used anywhere in the library.
// ---------------------------------------------------------------------------------------------
namespace harp {

void record_cuda_error(cudaError_t e);
void note_launch(int64_t k = 1);   // counts kernel launches (harp_launch_count)
// Streaming multiprocessors of the current device (queried once per device, then cached); every
// persistent grid and per-block scratch is sized from it.
int num_sms();
// Profiling: records an event closing segment `seg` (0..HARP_NSEGMENTS-1) on stream s when enabled.
enum : int { SEG_ORIENT = 0, SEG_TRI_WARP, SEG_TRI_CTA_S, SEG_TRI_CTA_L, SEG_TRI_FALLBACK, SEG_C4_SMALL,
             SEG_C4_MID, SEG_C4_WINDOW, SEG_REDUCE };
cudaError_t prof_mark(cudaStream_t s, int seg);

#define HARP_CK(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            ::harp::record_cuda_error(e_);             \
            return HARP_ECUDA;                         \
        }                                              \
    } while (0)

#define HARP_TRY(call)                                 \
    do {                                               \
        harp_status s_ = (call);                       \
        if (s_ != HARP_OK) return s_;                  \
    } while (0)

// after a <<<>>> launch
#define HARP_LAUNCHED()                                \
    do {                                               \
        ::harp::note_launch();                         \
        cudaError_t e_ = cudaGetLastError();           \
        if (e_ != cudaSuccess) {                       \
            ::harp::record_cuda_error(e_);             \
            return HARP_ECUDA;                         \
        }                                              \
    } while (0)

constexpr int kWarp = 32;
constexpr uint32_t kFull = 0xffffffffu;

// Slots of the device statistics / output vector (uint64[kOutLen]).
enum : int {
    OUT_COUNTS = 0,        // [0..5] induced counts
    OUT_STATS = 8,         // [8..15] HARP_STAT_* order
    ACC_T = 16,            // raw accumulators written by the kernels
    ACC_K4 = 17,
    ACC_C4 = 18,
    ACC_S = 19,            // sum_v C(d,3)
    ACC_PW = 20,           // sum_e (d_u-1)(d_v-1)
    ACC_PAWSUM = 21,       // sum over triangles of (d_a + d_b + d_c)
    ACC_D = 22,            // sum_e C(t_e, 2)
    ACC_M = 23,            // m
    ACC_ERR = 24,          // device-side consistency flags (0 = fine; kErr* bits)
    ACC_DONE = 25,         // last-block counter of the reduction kernel
    Q_TRI_WARP = 26,       // queue lengths
    Q_TRI_CTA = 27,
    Q_C4_MID = 28,
    Q_C4_WIN = 29,
    T_TRI_S = 30,          // work tickets of persistent kernels
    T_TRI_L = 31,
    T_TRI_F = 32,
    T_C4_MID = 33,
    T_C4_WIN = 34,
    W_TOTAL = 35,          // total window items of the windowed wedge kernel
    Q_SORT_CTA = 36,       // rows for the CTA row sort (36) and the hub row sort (37)
    T_TRI_M = 38,          // ticket of the 512-wide CTA triangle kernel
    ACC_SIG_HITS = 39,     // 4-clique extensions answered by a staged signature frontier
    Q_TRI_FB = 40,         // length of the unstaged-fallback triangle queue
    Q_TRI_BIG = 41,        // length of the global-staged triangle queue
    T_TRI_BIG = 42,        // its ticket
    // literal basis (Section III-F as printed): sums of the per-anchor terms; the three that are
    // divided (X_2 / 2, X_3 / 4, cycle pairs / 4) are 128-bit (lo, hi) so the division is exact
    ACC_LIT_X1 = 43,       // sum over triangles of X_1 (mod 2^64)
    ACC_LIT_X2 = 44,       // 44 lo, 45 hi
    ACC_LIT_X3 = 46,       // 46 lo, 47 hi
    ACC_LIT_AB = 48,       // sum over edges of |A_e| |B_e| (mod 2^64)
    ACC_LIT_E = 49,        // 49 lo, 50 hi: sum over edges of the A_e x B_e pairs that are edges
    ACC_LIT_STAR = 51,     // sum over vertices of the H_u star form (mod 2^64)
    ACC_LIT_T = 52,        // triangles enumerated by the literal triangle pass
    ACC_SIG_LOOKUPS = 53,  // literal basis: frontier requests to the signature cache
    Q_C4_MIDW = 54,        // length of the wedge middle tier's queue (from the back of q_mid)
    kOutLen = 64
};

// Bits of acc[ACC_ERR].  Any set bit makes a blocking count return HARP_EDEVICE; the asynchronous
// entry points copy the word to d_out[OUT_ERR].
constexpr uint64_t kErrSegment = 1;     // a wedge segment outside its window (skipped)
constexpr uint64_t kErrRow = 2;         // a wedge segment outside its row (skipped)
constexpr uint64_t kErrBadCsr = 256;    // a caller-built CSR failed its size/id check (nothing counted)
constexpr uint64_t kErrLitDiv = 512;    // a literal-closure sum was not divisible by its divisor
constexpr int OUT_ERR = 6;              // slot of d_out that receives acc[ACC_ERR]

// Per-graph accumulator slots (batch mode), kGStride per graph.
constexpr int kGStride = 8;
constexpr int kGInfo = 16;     // int64 per graph of wedge-window geometry
constexpr int kGridCap = 16;   // grid boundaries kept per row
enum : int { G_T = 0, G_K4, G_C4, G_S, G_PW, G_PAWSUM, G_D };

// ---------------------------------------------------------------------------------------------
// Workspace for one counting pass, sized for (n, m) and cached in the graph handle.
// ---------------------------------------------------------------------------------------------
struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    int64_t n = -1, m = -1;
    int32_t* deg = nullptr;        // [n]   degree in rank order
    int32_t* order = nullptr;      // [n]   new id -> old id
    int32_t* perm = nullptr;       // [n]   old id -> new id
    uint64_t* vkeys = nullptr;     // [n]   vertex sort keys
    uint64_t* vkeys_alt = nullptr; // [n]
    uint32_t* hist = nullptr;      // radix histograms
    size_t hist_len = 0;
    int64_t* off = nullptr;        // [n+1] rank-order CSR offsets
    int32_t* cols = nullptr;       // [2m]  rank-order CSR columns, rows ascending
    int32_t* dplus = nullptr;      // [n]   out-degree (neighbours with larger rank)
    int32_t* fpos = nullptr;       // [n]   first row position holding a neighbour of degree >= 2
    int32_t* rev = nullptr;        // [2m]  pos_w(u) for every lower arc (u -> w), at u's row position
    int32_t* bpos = nullptr;       // [n * kGridCap] row positions of the wedge-window grid boundaries
    int64_t* ginfo = nullptr;      // [G * kGInfo] per-graph bands of the wedge-window grid
    int64_t* offp = nullptr;       // [n+1] out-CSR offsets
    int32_t* colsp = nullptr;      // [m]   out-CSR columns
    uint32_t* te = nullptr;        // [m]   per out-arc triangle count t_e (colsp and te are contiguous)
    int32_t* q_tri = nullptr;      // [n]   CTA-mode triangle anchors
    int32_t* q_mid = nullptr;      // [n]   CTA-hash wedge roots
    int32_t* q_win = nullptr;      // [n]   windowed wedge roots
    int64_t* win_prefix = nullptr; // [n+1] window-item prefix over q_win
    int64_t* scan_tmp = nullptr;   // scan partials
    size_t scan_tmp_len = 0;
    uint64_t* acc = nullptr;       // [kOutLen]
    // batch mode only (the union of many graphs); nullptr for a single graph
    int64_t G = 1;                    // graphs
    const int64_t* gbase = nullptr;   // [G+1] first vertex of each graph (ranks and input ids alike)
    const int32_t* gid_in = nullptr;  // [n] graph of each input (union) vertex
    int32_t* gid = nullptr;           // [n] graph of each rank-order vertex
    uint64_t* accG = nullptr;         // [G * kGStride] per-graph accumulators
    // partitioned mode: only anchors/roots u in [own_lo, own_hi) are enumerated (the owner rule), and
    // the full-CSR arc count off[n] differs from 2m because halo rows are truncated (it may be 0);
    // -1 = a whole graph, off[n] = 2m
    int64_t own_lo = 0, own_hi = INT64_MAX;
    int64_t arcs = -1;
    // partitioned wedge pass: the roots' lower lists N-(u) in their own CSR (loff [n+1], lcols), the
    // rows (off, cols) hold only x in [x_lo, x_hi) (the opposite vertices this block owns); nullptr =
    // a whole graph, whose row prefixes are the lower lists.  bpos may be nullptr (window boundaries
    // are then searched in every row).
    const int64_t* loff = nullptr;
    const int32_t* lcols = nullptr;
    int64_t lower_arcs = 0;  // loff[n]
    int64_t x_lo = 0, x_hi = INT64_MAX;
};

// The workspace layout for (n, m): assigns every array of ws inside [base, base + returned bytes)
// (with base == nullptr it only computes the size).  Shared by every path that builds a workspace.
size_t ws_layout(Workspace& ws, unsigned char* base, int64_t n, int64_t m);
// stream-ordered allocation helpers
harp_status ws_ensure(Workspace& ws, int64_t n, int64_t m, cudaStream_t s);
void ws_release(Workspace& ws, cudaStream_t s);

}  // namespace harp

struct harp_csr {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0, m = 0, max_deg = 0;
    int64_t* off = nullptr;   // [n+1]
    int32_t* cols = nullptr;  // [2m]
    size_t csr_bytes = 0;
    harp::Workspace ws;
    // signature-reuse counters of the last blocking count (valid once have_reuse is set)
    uint64_t sig_lookups = 0, sig_hits = 0;
    bool have_reuse = false;
};

namespace harp {

// ---------------------------------------------------------------------------------------------
// Host launchers (one translation unit each).
// ---------------------------------------------------------------------------------------------

// scan.cu: out[i] = sum_{j<i} in[j] for i in [0, n]; out has n + 1 entries.
harp_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* tmp,
                                      size_t tmp_len, cudaStream_t s);
harp_status exclusive_scan_u32_inplace(uint32_t* data, int64_t n, int64_t* tmp, size_t tmp_len,
                                       cudaStream_t s);
size_t scan_tmp_needed(int64_t n);

// sort.cu: LSD radix sort of 64-bit keys on bits [begin_bit, end_bit); result ends in *keys
// (the pointer may be swapped with *alt).  hist needs radix_hist_len(n) entries.
harp_status radix_sort_u64(uint64_t** keys, uint64_t** alt, int64_t n, int begin_bit, int end_bit,
                           uint32_t* hist, int64_t* tmp, size_t tmp_len, cudaStream_t s);
size_t radix_hist_len(int64_t n);

// csr.cu
harp_status build_csr_device(harp_csr* g, int64_t n, int64_t m_in, const int32_t* d_src,
                             const int32_t* d_dst, cudaStream_t s);

// orient.cu: degree ordering + relabelled sorted CSR + out-CSR (step a1)
harp_status orient(const harp_csr* g, Workspace& ws, cudaStream_t s);

// tri.cu: triangle + per-edge t_e + 4-clique anchor (steps a3, a4)
harp_status count_triangles_k4(const harp_csr* g, Workspace& ws, const harp_plan& plan, cudaStream_t s);

// c4.cu: wedge anchor, non-induced 4-cycles (step a5)
harp_status count_wedge_c4(const harp_csr* g, Workspace& ws, const harp_plan& plan, cudaStream_t s);

// literal.cu: the literal basis (per-triangle X_j, per-edge A_e x B_e, per-vertex H_u stars) and its
// closure, after orient(); writes acc[OUT_COUNTS..], acc[OUT_STATS..]
harp_status count_literal(const harp_csr* g, Workspace& ws, const harp_plan& plan, cudaStream_t s);

// orbits.cu: per-vertex orbit counts (11 roles) after orient() and count_triangles_k4(); d_out is
// device uint64[n][11] indexed by input vertex id
harp_status count_orbits(const harp_csr* g, Workspace& ws, uint64_t* d_out, cudaStream_t s);
// per-edge orbit counts (10 roles); d_out is device uint64[m][10] in the input graph's edge order
harp_status count_edge_orbits(const harp_csr* g, Workspace& ws, uint64_t* d_out, cudaStream_t s);

// reduce.cu: sum_e C(t_e,2), closure (step a7); writes acc[OUT_COUNTS..], acc[OUT_STATS..]
harp_status reduce_and_close(const harp_csr* g, Workspace& ws, cudaStream_t s);
// batch mode: per-graph sum_e C(t_e,2) and closure; d_out holds 16 uint64 per graph
harp_status reduce_and_close_batch(const harp_csr* g, Workspace& ws, int64_t G, uint64_t* d_out, cudaStream_t s);

// planner.cu
void default_plan(harp_plan* p);
void normalise_plan(const harp_plan* in, harp_plan* out);
// Bytes of a caller's plan that are read: version-1 plans end at `objective`.
size_t plan_bytes(const harp_plan* p);

// ---------------------------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Block-wide sum of a uint64 (all threads participate; result valid in thread 0).
__device__ __forceinline__ uint64_t block_sum_u64(uint64_t v, uint64_t* smem32) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) smem32[w] = v;
    __syncthreads();
    uint64_t r = 0;
    if (threadIdx.x < 32) {
        const int nw = (blockDim.x + 31) >> 5;
        r = (threadIdx.x < nw) ? smem32[threadIdx.x] : 0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Where anchor statistics go.  Single graph: thread-local sums, one block reduction and one atomic
// per block at the end (acc[ACC_*]).  Batch (the disjoint union of many graphs): every anchor's sum
// goes to its own graph's slot accG[gid[anchor] * kGStride + G_*] as soon as the anchor is done.
struct Sink {
    uint64_t* acc;
    const int32_t* gid;
    uint64_t* accG;
    __device__ __forceinline__ bool batch() const { return gid != nullptr; }
};

__device__ __forceinline__ void sink_add(const Sink& s, int32_t anchor, int gslot, uint64_t v) {
    if (v) atomicAdd((unsigned long long*)&s.accG[(int64_t)s.gid[anchor] * kGStride + gslot],
                     (unsigned long long)v);
}

// lower_bound in a sorted int32 array a[0..len): first index with a[i] >= key
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t len, int32_t key) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) { return x * 0x9E3779B1u; }

// C(x, 2) and C(x, 3) exactly modulo 2^64 (the divisor is removed from a factor first)
__device__ __forceinline__ uint64_t choose2_u64(uint64_t x) {
    if (x < 2) return 0;
    uint64_t a = x, b = x - 1;
    if ((a & 1) == 0) a >>= 1; else b >>= 1;
    return a * b;
}
__device__ __forceinline__ uint64_t choose3_u64(uint64_t x) {
    if (x < 3) return 0;
    uint64_t f0 = x, f1 = x - 1, f2 = x - 2;
    if (f0 % 3 == 0) f0 /= 3; else if (f1 % 3 == 0) f1 /= 3; else f2 /= 3;
    if ((f0 & 1) == 0) f0 >>= 1; else if ((f1 & 1) == 0) f1 >>= 1; else f2 >>= 1;
    return f0 * f1 * f2;
}

}  // namespace harp
