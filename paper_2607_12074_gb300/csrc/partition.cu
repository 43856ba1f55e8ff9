// Step a9: ownership-preserving partitioned counting (Section III-E) for graphs whose counting
// footprint exceeds a device-memory budget.
//
// The host builds the simple graph in global rank order (rank = (degree, id)) and cuts the rank
// space into contiguous ranges P_k sized to the budget.  The canonical owner certificate of an anchor
// is the partition of the first vertex of its globally ordered anchor tuple: a triangle / 4-clique
// anchor and all its per-edge contributions belong to its lowest vertex u, a wedge (4-cycle) anchor
// to its top vertex u.  Partition k enumerates exactly the anchors it owns, over a halo that holds
// every row those anchors read:
//   * rows of u in P_k and of every lower neighbour w of such u, truncated to entries below P_k's
//     upper bound (the wedge prefixes x < u and the lower lists N-(u) lie inside; a truncation only
//     drops a row's suffix, so every row position used by the kernels equals the global one);
//   * the out-lists N+(v) of every vertex v in P_k or adjacent to one (triangle intersections, the
//     position of u in N+(w)).
// Replicated halo rows therefore serve completion checks without contributing counts.  Sums of
// anchor statistics are additive over partitions; per-edge triangle counts t_e receive contributions
// from several partitions and are summed into one global array before sum_e C(t_e, 2) is formed.
// The degree sums and the closure are evaluated once at the end, so every count is exact.
#include <algorithm>
#include <cstring>
#include <utility>
#include <new>
#include <thread>
#include <vector>

#include "harp_internal.cuh"

namespace harp {
namespace {

// LSD radix sort of 64-bit keys on the host (16-bit digits over the significant bits), threads split
// every pass by contiguous slices so the sort stays stable.
void host_radix_sort(std::vector<uint64_t>& a, int bits) {
    const size_t n = a.size();
    if (n < 2 || bits <= 0) return;
    std::vector<uint64_t> b(n);
    unsigned nt = std::thread::hardware_concurrency();
    if (nt < 1) nt = 1;
    if (nt > 64) nt = 64;
    if (n < (size_t)1 << 16) nt = 1;
    const int digit = 16;
    std::vector<std::vector<size_t>> hist(nt, std::vector<size_t>((size_t)1 << digit));
    for (int shift = 0; shift < bits; shift += digit) {
        const uint64_t mask = ((uint64_t)1 << digit) - 1;
        auto slice = [&](unsigned t, size_t& lo, size_t& hi) {
            lo = n * t / nt;
            hi = n * (t + 1) / nt;
        };
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                size_t lo, hi;
                slice(t, lo, hi);
                std::fill(hist[t].begin(), hist[t].end(), 0);
                for (size_t i = lo; i < hi; ++i) hist[t][(a[i] >> shift) & mask]++;
            });
        for (auto& x : th) x.join();
        th.clear();
        size_t run = 0;
        for (size_t d = 0; d < ((size_t)1 << digit); ++d)
            for (unsigned t = 0; t < nt; ++t) {
                const size_t c = hist[t][d];
                hist[t][d] = run;
                run += c;
            }
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                size_t lo, hi;
                slice(t, lo, hi);
                std::vector<size_t>& h = hist[t];
                for (size_t i = lo; i < hi; ++i) b[h[(a[i] >> shift) & mask]++] = a[i];
            });
        for (auto& x : th) x.join();
        a.swap(b);
    }
}

int bits_of(uint64_t x) {
    int b = 0;
    while (b < 64 && ((uint64_t)1 << b) <= x) ++b;
    return b < 1 ? 1 : b;
}

// The simple graph in global rank order: symmetric CSR with sorted rows (host memory).
struct RankGraph {
    int64_t n = 0, m = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> cols;
    std::vector<int32_t> deg, dplus;  // by rank
    std::vector<int64_t> offp;        // out-arc numbering: N+(r) holds global out-arcs offp[r] ..
};

harp_status build_rank_graph(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, RankGraph& g) {
    std::vector<uint64_t> keys;
    keys.reserve((size_t)m_in);
    const int b = bits_of((uint64_t)n);
    for (int64_t e = 0; e < m_in; ++e) {
        const int32_t u = src[e], v = dst[e];
        if (u < 0 || v < 0 || u >= n || v >= n) return HARP_EINVAL;
        if (u == v) continue;
        const uint64_t lo = (uint64_t)(u < v ? u : v), hi = (uint64_t)(u < v ? v : u);
        keys.push_back((lo << b) | hi);
    }
    host_radix_sort(keys, 2 * b);
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    g.n = n;
    g.m = (int64_t)keys.size();
    const uint64_t lowmask = ((uint64_t)1 << b) - 1;
    std::vector<int32_t> deg0((size_t)n, 0);
    for (uint64_t k : keys) {
        deg0[k >> b]++;
        deg0[k & lowmask]++;
    }
    // rank = (degree, id): counting sort by degree, ids ascending inside a degree
    int32_t maxd = 0;
    for (int32_t d : deg0) maxd = d > maxd ? d : maxd;
    std::vector<int64_t> start((size_t)maxd + 2, 0);
    for (int32_t d : deg0) start[(size_t)d + 1]++;
    for (size_t d = 0; d + 1 < start.size(); ++d) start[d + 1] += start[d];
    std::vector<int32_t> rank((size_t)n);
    for (int64_t v = 0; v < n; ++v) rank[(size_t)v] = (int32_t)start[(size_t)deg0[(size_t)v]]++;
    std::vector<uint64_t> arcs;
    arcs.reserve(2 * keys.size());
    for (uint64_t k : keys) {
        const uint64_t a = (uint64_t)rank[k >> b], c = (uint64_t)rank[k & lowmask];
        arcs.push_back((a << 32) | c);
        arcs.push_back((c << 32) | a);
    }
    std::vector<uint64_t>().swap(keys);
    host_radix_sort(arcs, 32 + b);
    g.off.assign((size_t)n + 1, 0);
    g.cols.resize(arcs.size());
    for (size_t i = 0; i < arcs.size(); ++i) {
        g.off[(arcs[i] >> 32) + 1]++;
        g.cols[i] = (int32_t)(arcs[i] & 0xffffffffull);
    }
    for (int64_t r = 0; r < n; ++r) g.off[(size_t)r + 1] += g.off[(size_t)r];
    g.deg.resize((size_t)n);
    g.dplus.resize((size_t)n);
    g.offp.assign((size_t)n + 1, 0);
    for (int64_t r = 0; r < n; ++r) {
        const int64_t lo = g.off[(size_t)r], hi = g.off[(size_t)r + 1];
        g.deg[(size_t)r] = (int32_t)(hi - lo);
        const int64_t split = std::upper_bound(g.cols.begin() + lo, g.cols.begin() + hi, (int32_t)r) -
                              (g.cols.begin() + lo);
        g.dplus[(size_t)r] = (int32_t)(hi - lo - split);
        g.offp[(size_t)r + 1] = g.offp[(size_t)r] + g.dplus[(size_t)r];
    }
    return HARP_OK;
}

uint64_t choose2_h(uint64_t x) {
    if (x < 2) return 0;
    uint64_t a = x, b = x - 1;
    if (a % 2 == 0) a /= 2; else b /= 2;
    return a * b;
}

uint64_t choose3_h(uint64_t x) {
    if (x < 3) return 0;
    uint64_t f[3] = {x, x - 1, x - 2};
    for (int i = 0; i < 3; ++i) if (f[i] % 3 == 0) { f[i] /= 3; break; }
    for (int i = 0; i < 3; ++i) if (f[i] % 2 == 0) { f[i] /= 2; break; }
    return f[0] * f[1] * f[2];
}

// One partition's halo, laid out like the kernels' rank-order arrays (global ids, empty rows for
// vertices outside the halo).
struct Halo {
    std::vector<int64_t> off, offp;
    std::vector<int32_t> cols, colsp;
    std::vector<int64_t> gpos;  // for every local out-arc row start: global out-arc id of N+(v)[0]
};

void build_halo(const RankGraph& g, int64_t lo, int64_t hi, Halo& h) {
    const int64_t n = g.n;
    std::vector<uint8_t> inH((size_t)n, 0), inO((size_t)n, 0);
    for (int64_t u = lo; u < hi; ++u) {
        inH[(size_t)u] = 1;
        inO[(size_t)u] = 1;
        for (int64_t a = g.off[(size_t)u]; a < g.off[(size_t)u + 1]; ++a) {
            const int32_t x = g.cols[(size_t)a];
            inO[(size_t)x] = 1;             // neighbours: their out-lists (both directions)
            if (x < u) inH[(size_t)x] = 1;  // lower neighbours: their rows (wedge prefixes)
        }
    }
    h.off.assign((size_t)n + 1, 0);
    h.offp.assign((size_t)n + 1, 0);
    for (int64_t v = 0; v < n; ++v) {
        int64_t len = 0;
        if (inH[(size_t)v]) {
            const auto b = g.cols.begin() + g.off[(size_t)v], e = g.cols.begin() + g.off[(size_t)v + 1];
            len = std::lower_bound(b, e, (int32_t)hi) - b;  // truncated below the range's upper bound
        }
        h.off[(size_t)v + 1] = h.off[(size_t)v] + len;
        h.offp[(size_t)v + 1] = h.offp[(size_t)v] + (inO[(size_t)v] ? g.dplus[(size_t)v] : 0);
    }
    h.cols.resize((size_t)h.off[(size_t)n]);
    h.colsp.resize((size_t)h.offp[(size_t)n]);
    for (int64_t v = 0; v < n; ++v) {
        const int64_t len = h.off[(size_t)v + 1] - h.off[(size_t)v];
        if (len) std::memcpy(&h.cols[(size_t)h.off[(size_t)v]], &g.cols[(size_t)g.off[(size_t)v]], sizeof(int32_t) * (size_t)len);
        const int64_t lp = h.offp[(size_t)v + 1] - h.offp[(size_t)v];
        if (lp)
            std::memcpy(&h.colsp[(size_t)h.offp[(size_t)v]], &g.cols[(size_t)(g.off[(size_t)v + 1] - lp)],
                        sizeof(int32_t) * (size_t)lp);
    }
}

// Device bytes a partition with this many halo arcs and out-arcs needs (the layout the counting
// kernels use).
size_t halo_bytes(int64_t n, int64_t arcs, int64_t out_arcs) {
    Workspace probe;
    const int64_t mws = std::max((arcs + 1) / 2, out_arcs);
    return ws_layout(probe, nullptr, n, mws);
}

// The size of build_halo's result for [lo, hi) without copying it: (row arcs, out-arcs).  Monotone in
// hi for a fixed lo (a longer range adds rows and raises the truncation bound).
std::pair<int64_t, int64_t> halo_extent(const RankGraph& g, int64_t lo, int64_t hi, std::vector<uint8_t>& inH,
                                        std::vector<uint8_t>& inO, std::vector<int32_t>& touched) {
    touched.clear();
    auto mark = [&](std::vector<uint8_t>& f, int32_t v, uint8_t bit) {
        if (!(inH[(size_t)v] | inO[(size_t)v])) touched.push_back(v);
        f[(size_t)v] |= bit;
    };
    for (int64_t u = lo; u < hi; ++u) {
        mark(inH, (int32_t)u, 1);
        mark(inO, (int32_t)u, 1);
        for (int64_t a = g.off[(size_t)u]; a < g.off[(size_t)u + 1]; ++a) {
            const int32_t x = g.cols[(size_t)a];
            mark(inO, x, 1);
            if (x < u) mark(inH, x, 1);
        }
    }
    int64_t arcs = 0, outs = 0;
    for (int32_t v : touched) {
        if (inH[(size_t)v]) {
            const auto b = g.cols.begin() + g.off[(size_t)v], e = g.cols.begin() + g.off[(size_t)v + 1];
            arcs += std::lower_bound(b, e, (int32_t)hi) - b;
        }
        if (inO[(size_t)v]) outs += g.dplus[(size_t)v];
        inH[(size_t)v] = inO[(size_t)v] = 0;
    }
    return {arcs, outs};
}

}  // namespace
}  // namespace harp

using namespace harp;

extern "C" harp_status harp_count4_partitioned(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                                               uint64_t budget_bytes, int32_t parts, uint64_t counts_out[6],
                                               harp_partition_stats* stats) {
    if (!counts_out || n < 0 || m_in < 0 || (m_in > 0 && (!src || !dst)) || parts < 0) return HARP_EINVAL;
    if (n > 2147483647LL || m_in > 2147483647LL) return HARP_EOVERFLOW;
    int dev = 0;
    HARP_CK(cudaGetDevice(&dev));
    RankGraph g;
    HARP_TRY(build_rank_graph(n, m_in, src, dst, g));
    if (budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        HARP_CK(cudaMemGetInfo(&fr, &tot));
        budget_bytes = fr / 2;
    }
    // Cut rank space into ranges: a fixed count if asked, otherwise greedily, each range the longest
    // whose halo fits the budget (binary search; the halo size is monotone in the range's end).  A
    // single vertex whose halo exceeds the budget cannot be counted under it: HARP_ENOMEM.
    std::vector<int64_t> cuts{0};
    if (parts > 0) {
        for (int32_t k = 1; k < parts; ++k) cuts.push_back(n * k / parts);
        cuts.push_back(n);
    } else {
        std::vector<uint8_t> inH((size_t)n, 0), inO((size_t)n, 0);
        std::vector<int32_t> touched;
        auto fits = [&](int64_t lo, int64_t hi) {
            const auto ext = halo_extent(g, lo, hi, inH, inO, touched);
            return halo_bytes(n, ext.first, ext.second) <= budget_bytes;
        };
        int64_t lo = 0;
        while (lo < n) {
            if (!fits(lo, lo + 1)) return HARP_ENOMEM;
            int64_t good = lo + 1, bad = n + 1;  // fits(lo, good) holds; fits(lo, bad) does not (n + 1: none)
            if (fits(lo, n)) good = n;
            else bad = n;
            while (bad - good > 1) {
                const int64_t mid = good + (bad - good) / 2;
                if (fits(lo, mid)) good = mid;
                else bad = mid;
            }
            cuts.push_back(good);
            lo = good;
        }
    }
    std::vector<uint32_t> te_global((size_t)g.offp[(size_t)n], 0);
    uint64_t T = 0, K4 = 0, C4 = 0, PAWSUM = 0;
    uint64_t host_bytes = 0, device_peak = 0, halo_arcs = 0;
    cudaStream_t s = nullptr;
    HARP_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    harp_status st = HARP_OK;
    for (size_t k = 0; k + 1 < cuts.size() && st == HARP_OK; ++k) {
        const int64_t lo = cuts[k], hi = cuts[k + 1];
        if (lo >= hi) continue;
        Halo h;
        build_halo(g, lo, hi, h);
        const int64_t arcs = (int64_t)h.cols.size(), out_arcs = (int64_t)h.colsp.size();
        halo_arcs += (uint64_t)(arcs + out_arcs);
        const int64_t mws = std::max((arcs + 1) / 2, out_arcs);
        Workspace probe;
        const size_t bytes = ws_layout(probe, nullptr, n, mws);
        if (bytes > device_peak) device_peak = bytes;
        void* base = nullptr;
        cudaError_t e = cudaMallocAsync(&base, bytes, s);
        if (e != cudaSuccess) {
            record_cuda_error(e);
            st = e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
            break;
        }
        Workspace ws;
        ws_layout(ws, static_cast<unsigned char*>(base), n, mws);
        ws.own_lo = lo;
        ws.own_hi = hi;
        ws.arcs = arcs;
        // host -> device: the halo and the global degree arrays (the transfer Table IV measures)
        e = cudaMemcpyAsync(ws.off, h.off.data(), sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && arcs)
            e = cudaMemcpyAsync(ws.cols, h.cols.data(), sizeof(int32_t) * (size_t)arcs, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws.offp, h.offp.data(), sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && out_arcs)
            e = cudaMemcpyAsync(ws.colsp, h.colsp.data(), sizeof(int32_t) * (size_t)out_arcs, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws.deg, g.deg.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws.dplus, g.dplus.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ws.te, 0, sizeof(uint32_t) * (size_t)(out_arcs > 0 ? out_arcs : 1), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s);
        host_bytes += 8 * (uint64_t)(n + 1) * 2 + 4 * (uint64_t)(arcs + out_arcs) + 8 * (uint64_t)n;
        if (e != cudaSuccess) {
            record_cuda_error(e);
            st = HARP_ECUDA;
        }
        harp_csr view;  // the kernels' view: global n and m (m sizes the hub fallback), halo arrays
        view.device = dev;
        view.stream = s;
        view.n = n;
        view.m = g.m;
        int32_t maxd = 0;
        for (int32_t d : g.deg) maxd = d > maxd ? d : maxd;
        view.max_deg = maxd;
        view.off = ws.off;
        view.cols = ws.cols;
        harp_plan plan;
        normalise_plan(nullptr, &plan);
        if (st == HARP_OK && n > 0) st = count_triangles_k4(&view, ws, plan, s);
        if (st == HARP_OK && n > 0) st = count_wedge_c4(&view, ws, plan, s);
        std::vector<uint32_t> te_local((size_t)out_arcs);
        uint64_t acc[kOutLen];
        if (st == HARP_OK) {
            e = cudaMemcpyAsync(acc, ws.acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && out_arcs)
                e = cudaMemcpyAsync(te_local.data(), ws.te, sizeof(uint32_t) * (size_t)out_arcs, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                record_cuda_error(e);
                st = HARP_ECUDA;
            } else if (acc[ACC_ERR]) {
                st = HARP_EDEVICE;
            }
        }
        cudaFreeAsync(base, s);
        if (st != HARP_OK) break;
        T += acc[ACC_T];
        K4 += acc[ACC_K4];
        C4 += acc[ACC_C4];
        PAWSUM += acc[ACC_PAWSUM];
        for (int64_t v = 0; v < n; ++v) {  // local out-arcs -> global out-arc ids
            const int64_t lb = h.offp[(size_t)v], len = h.offp[(size_t)v + 1] - lb;
            const int64_t gb = g.offp[(size_t)v];
            for (int64_t k2 = 0; k2 < len; ++k2) te_global[(size_t)(gb + k2)] += te_local[(size_t)(lb + k2)];
        }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (st != HARP_OK) return st;
    // degree sums by owner (every vertex / edge once) and the global sum_e C(t_e, 2)
    uint64_t S = 0, PW = 0, D = 0;
    for (int64_t r = 0; r < n; ++r) {
        const uint64_t dr = (uint64_t)g.deg[(size_t)r];
        S += choose3_h(dr);
        for (int64_t a = g.off[(size_t)r + 1] - g.dplus[(size_t)r]; a < g.off[(size_t)r + 1]; ++a)
            PW += (dr - 1) * ((uint64_t)g.deg[(size_t)g.cols[(size_t)a]] - 1);
    }
    for (uint32_t t : te_global) D += choose2_h(t);
    const uint64_t P = PW - 3 * T, pawn = PAWSUM - 6 * T;
    const uint64_t diamond = D - 6 * K4;
    const uint64_t c4 = C4 - diamond - 3 * K4;
    const uint64_t paw = pawn - 4 * diamond - 12 * K4;
    const uint64_t path = P - 2 * paw - 4 * c4 - 6 * diamond - 12 * K4;
    const uint64_t star = S - paw - 2 * diamond - 4 * K4;
    counts_out[HARP_STAR3] = star;
    counts_out[HARP_PATH4] = path;
    counts_out[HARP_PAW] = paw;
    counts_out[HARP_CYCLE4] = c4;
    counts_out[HARP_DIAMOND] = diamond;
    counts_out[HARP_CLIQUE4] = K4;
    if (stats) {
        stats->partitions = (int64_t)cuts.size() - 1;
        stats->m = g.m;
        stats->halo_arcs = (int64_t)halo_arcs;
        stats->h2d_bytes = host_bytes;
        stats->device_peak_bytes = device_peak;
    }
    return HARP_OK;
}
