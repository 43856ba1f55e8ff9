// Step a9: ownership-preserving partitioned counting (Section III-E) for graphs whose counting
// footprint exceeds a device-memory budget.
//
// The host builds the simple graph in global rank order (rank = (degree, id)).  Every anchor has a
// canonical owner certificate taken from its globally ordered tuple, and each device block counts
// exactly the anchors it owns over a halo that holds every list those anchors read:
//   * triangle / 4-clique / t_e anchors {u < v < w} belong to the rank range of u.  A triangle block
//     for the range R holds the out-lists N+(v) of every v in R or in N+(R) (1 hop) and their t_e.
//   * wedge (4-cycle) anchors (u top, x opposite, both middles below u) belong to the pair (rank range
//     of u, x-slice of x): Sum_x C(cnt(x), 2) is additive over disjoint slices of x.  A wedge block
//     for (R, X) holds the lower lists N-(u) of the roots u in R and, for every lower neighbour w of
//     such a root, the part of w's row inside X below R's end (2 hops through lower-ranked vertices).
// Replicated halo lists serve completion checks without contributing counts.  Per-edge triangle
// counts t_e receive contributions from several triangle blocks and are summed into one global
// array before Sum_e C(t_e, 2); the degree sums and the closure are evaluated once at the end, so
// every count is exact.  Ranges are cut by one linear sweep each, as long as the exact halo size
// fits the budget; a single vertex (or x-value) whose halo does not fit gives HARP_ENOMEM.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "harp_internal.cuh"

namespace harp {
namespace {

unsigned host_threads() {
    unsigned nt = std::thread::hardware_concurrency();
    return nt < 1 ? 1 : (nt > 64 ? 64 : nt);
}

// f(lo, hi, t) over contiguous slices of [0, n), one per host thread (inline when n is small).
template <typename F>
void parallel_for(int64_t n, F&& f) {
    const unsigned nt = n < (1 << 16) ? 1 : host_threads();
    if (nt == 1) {
        f((int64_t)0, n, 0u);
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] { f(n * (int64_t)t / (int64_t)nt, n * (int64_t)(t + 1) / (int64_t)nt, t); });
    for (auto& x : th) x.join();
}

// Allocator whose resize leaves new elements uninitialised: multi-gigabyte arrays that are written in
// full right after (rows, halo copies, device read-backs) are not zero-filled first on one core.
template <typename T>
struct NoInit : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = NoInit<U>;
    };
    NoInit() = default;
    template <typename U>
    NoInit(const NoInit<U>&) {}
    template <typename U>
    void construct(U*) noexcept {}
    template <typename U, typename... A>
    void construct(U* p, A&&... a) {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
};
template <typename T>
using buf = std::vector<T, NoInit<T>>;

// The simple graph in global rank order: symmetric CSR with sorted rows (host memory).
struct RankGraph {
    int64_t n = 0, m = 0;
    std::vector<int64_t> off;
    buf<int32_t> cols;
    std::vector<int32_t> deg, dplus;  // by rank
    std::vector<int64_t> offp;        // global out-arc numbering: N+(r) holds out-arcs offp[r] ..
    int64_t n1 = 0;                   // first rank of degree >= 2
    std::vector<int32_t> rank;        // rank[v] of input vertex v
};

// f(lo, hi) over chunks of [0, n) taken from a shared counter by every host thread (rows of very
// different lengths, e.g. hubs at the start of the id range, stay balanced).
template <typename F>
void parallel_dynamic(int64_t n, int64_t chunk, F&& f) {
    const unsigned nt = (n + chunk - 1) / chunk < 2 ? 1 : host_threads();
    std::atomic<int64_t> next{0};
    auto run = [&] {
        for (;;) {
            const int64_t lo = next.fetch_add(chunk);
            if (lo >= n) return;
            f(lo, lo + chunk < n ? lo + chunk : n);
        }
    };
    if (nt == 1) {
        run();
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) th.emplace_back(run);
    for (auto& x : th) x.join();
}

// Stable regrouping of a symmetric arc multiset by its other endpoint.  Sources i = 0 .. N - 1 are
// visited in increasing order; source i's entries are row(i) = [begin, end) of `cols`.  Entry c of
// source i goes to destination row dest(c) with value i, so every destination row receives its
// values in increasing order (sorted rows without a sort).  out_off[0 .. n_dest] are the destination
// rows' offsets; because the arcs are symmetric they are also the prefix of the sources' entry counts
// in visit order, which balances the sources over the host threads.  scratch holds out_off[n_dest]
// packed (row, value) pairs.  Every source row is read before the first value is placed, so `out`
// may be the buffer the source rows live in.
// done(d0, d1) runs on destination rows [d0, d1) right after they are filled (while they are in cache).
constexpr int64_t kRegroupBuckets = 4096;
template <typename RowOf, typename DestOf, typename Done>
void regroup_by_destination(int64_t N, RowOf row, DestOf dest, int64_t n_dest, const int64_t* out_off, int32_t* out,
                            uint64_t* scratch, Done&& done) {
    int sh = 0;  // destination bucket: d >> sh, about kRegroupBuckets buckets
    while ((n_dest >> sh) > kRegroupBuckets) ++sh;
    const int64_t nb = (n_dest >> sh) + 1;
    const int64_t total = out_off[n_dest];
    const unsigned nt = total < (1 << 16) ? 1 : host_threads();
    std::vector<int64_t> cut((size_t)nt + 1, N);  // thread t visits sources [cut[t], cut[t+1])
    cut[0] = 0;
    for (unsigned t = 1; t < nt; ++t)
        cut[t] = std::upper_bound(out_off, out_off + N + 1, total * (int64_t)t / (int64_t)nt) - out_off - 1;
    for (unsigned t = 1; t <= nt; ++t) cut[t] = std::max(cut[t], cut[t - 1]);
    std::vector<std::vector<int64_t>> cnt(nt, std::vector<int64_t>((size_t)nb, 0));
    auto each_thread = [&](auto&& f) {
        if (nt == 1) {
            f(0u);
            return;
        }
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) th.emplace_back([&, t] { f(t); });
        for (auto& x : th) x.join();
    };
    each_thread([&](unsigned t) {
        std::vector<int64_t>& c = cnt[t];
        for (int64_t i = cut[t]; i < cut[t + 1]; ++i) {
            const auto r = row(i);
            for (const int32_t* p = r.first; p != r.second; ++p) c[(size_t)(dest(*p) >> sh)]++;
        }
    });
    std::vector<int64_t> bstart((size_t)nb + 1, 0);
    for (int64_t k = 0; k < nb; ++k) {  // bucket k, thread t's part after those of threads < t
        int64_t run = bstart[(size_t)k];
        for (unsigned t = 0; t < nt; ++t) {
            const int64_t c = cnt[t][(size_t)k];
            cnt[t][(size_t)k] = run;
            run += c;
        }
        bstart[(size_t)k + 1] = run;
    }
    each_thread([&](unsigned t) {
        std::vector<int64_t>& cur = cnt[t];
        for (int64_t i = cut[t]; i < cut[t + 1]; ++i) {
            const auto r = row(i);
            for (const int32_t* p = r.first; p != r.second; ++p) {
                const int64_t d = dest(*p);
                scratch[(size_t)cur[(size_t)(d >> sh)]++] = ((uint64_t)d << 32) | (uint32_t)i;
            }
        }
    });
    parallel_dynamic(nb, 1, [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t d0 = k << sh, d1 = std::min<int64_t>((k + 1) << sh, n_dest);
            if (d0 >= d1) continue;
            std::vector<int64_t> pos((size_t)(d1 - d0));
            for (int64_t d = d0; d < d1; ++d) pos[(size_t)(d - d0)] = out_off[d];
            for (int64_t e = bstart[(size_t)k]; e < bstart[(size_t)k + 1]; ++e) {
                const uint64_t pr = scratch[(size_t)e];
                const int64_t d = (int64_t)(pr >> 32);
                out[pos[(size_t)(d - d0)]++] = (int32_t)(uint32_t)pr;
            }
            done(d0, d1);
        }
    });
}

// The rank-order CSR without atomics and without sorting rows: arcs are partitioned by source-id
// bucket (per-thread histograms and thread-private cursors), each bucket is turned into its rows and
// each row's duplicates are dropped through a hash table; the rank order (degree, id) is a counting
// sort by degree; regrouping the rows by their other endpoint, relabelled, with vertices visited in
// rank order, gives rows sorted by rank.
harp_status build_rank_graph(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, RankGraph& g) {
    int sh = 0;  // bucket of a vertex: v >> sh, about 1024 buckets
    while ((n >> sh) > 1024) ++sh;
    const int64_t nb = (n >> sh) + 1;
    const unsigned nt = m_in < (1 << 16) ? 1 : host_threads();
    std::vector<std::vector<int64_t>> hist(nt, std::vector<int64_t>((size_t)nb, 0));
    std::vector<uint8_t> bad(nt, 0);
    auto slice = [&](unsigned t, int64_t& lo, int64_t& hi) {
        lo = m_in * (int64_t)t / (int64_t)nt;
        hi = m_in * (int64_t)(t + 1) / (int64_t)nt;
    };
    {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                int64_t lo, hi;
                slice(t, lo, hi);
                std::vector<int64_t>& h = hist[t];
                for (int64_t e = lo; e < hi; ++e) {
                    const int32_t u = src[e], v = dst[e];
                    if (u < 0 || v < 0 || u >= n || v >= n) {
                        bad[t] = 1;
                        continue;
                    }
                    if (u == v) continue;
                    h[(size_t)(u >> sh)]++;
                    h[(size_t)(v >> sh)]++;
                }
            });
        for (auto& x : th) x.join();
    }
    for (uint8_t x : bad)
        if (x) return HARP_EINVAL;
    std::vector<int64_t> bstart((size_t)nb + 1, 0);
    for (int64_t k = 0; k < nb; ++k) {  // bucket k: [bstart[k], bstart[k+1]); thread t's part in order
        int64_t run = bstart[(size_t)k];
        for (unsigned t = 0; t < nt; ++t) {
            const int64_t c = hist[t][(size_t)k];
            hist[t][(size_t)k] = run;
            run += c;
        }
        bstart[(size_t)k + 1] = run;
    }
    const int64_t A = bstart[(size_t)nb];
    buf<uint64_t> pairs;  // (row << 32) | column, in bucket order; later the regrouping scratch
    // The rows, in one buffer throughout: by id with duplicates, by id without, relabelled, then by
    // rank (the regrouping reads its input rows before it places a value).
    buf<int32_t> c0;
    try {
        pairs.resize((size_t)(A > 0 ? A : 1));
        c0.resize((size_t)(A > 0 ? A : 1));
    } catch (...) {
        return HARP_ENOMEM;
    }
    {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                int64_t lo, hi;
                slice(t, lo, hi);
                std::vector<int64_t>& cur = hist[t];
                for (int64_t e = lo; e < hi; ++e) {
                    const int32_t u = src[e], v = dst[e];
                    if (u == v) continue;
                    pairs[(size_t)cur[(size_t)(u >> sh)]++] = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
                    pairs[(size_t)cur[(size_t)(v >> sh)]++] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)u;
                }
            });
        for (auto& x : th) x.join();
    }
    std::vector<std::vector<int64_t>>().swap(hist);
    // each bucket into its rows (positions of the id-order CSR are the bucket's own range), then each
    // row's duplicates dropped in place through a small hash table (stamped by row, so it is never
    // cleared): row v keeps deg0[v] entries from off0[v], in first-seen order
    std::vector<int64_t> off0((size_t)n + 1, 0);
    std::vector<int32_t> deg0((size_t)n, 0);
    parallel_dynamic(nb, 1, [&](int64_t k0, int64_t k1) {
        thread_local std::vector<uint64_t> table;
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t r0 = k << sh, r1 = std::min<int64_t>((k + 1) << sh, n);
            if (r0 >= r1) continue;
            std::vector<int64_t> pos((size_t)(r1 - r0 + 1), 0);
            for (int64_t i = bstart[(size_t)k]; i < bstart[(size_t)k + 1]; ++i)
                pos[(size_t)((int64_t)(pairs[(size_t)i] >> 32) - r0) + 1]++;
            for (int64_t r = 0; r < r1 - r0; ++r) pos[(size_t)r + 1] += pos[(size_t)r];
            for (int64_t r = r0; r < r1; ++r) off0[(size_t)r] = bstart[(size_t)k] + pos[(size_t)(r - r0)];
            for (int64_t i = bstart[(size_t)k]; i < bstart[(size_t)k + 1]; ++i) {
                const uint64_t pr = pairs[(size_t)i];
                c0[(size_t)(bstart[(size_t)k] + pos[(size_t)((int64_t)(pr >> 32) - r0)]++)] = (int32_t)(uint32_t)pr;
            }
            for (int64_t r = r0; r < r1; ++r) {  // after the scatter pos[r - r0] is the end of row r
                const int64_t beg = off0[(size_t)r], end = bstart[(size_t)k] + pos[(size_t)(r - r0)];
                if (end - beg <= 1) {
                    deg0[(size_t)r] = (int32_t)(end - beg);
                    continue;
                }
                int lg = 1;
                while (((int64_t)1 << lg) < 2 * (end - beg)) ++lg;
                if (table.size() < ((size_t)1 << lg)) table.assign((size_t)1 << lg, 0);  // stamp 0: empty
                const uint64_t stamp = (uint64_t)(r + 1) << 32, mask = ((uint64_t)1 << lg) - 1;
                int64_t w = beg;
                for (int64_t i = beg; i < end; ++i) {
                    const uint32_t v = (uint32_t)c0[(size_t)i];
                    uint64_t h = ((uint64_t)v * 0x9E3779B97F4A7C15ull) >> (64 - lg);
                    for (;;) {
                        const uint64_t e = table[(size_t)h];
                        if ((e & ~0xffffffffull) != stamp) {  // a slot of another row: free here
                            table[(size_t)h] = stamp | v;
                            c0[(size_t)w++] = (int32_t)v;
                            break;
                        }
                        if ((uint32_t)e == v) break;  // a duplicate
                        h = (h + 1) & mask;
                    }
                }
                deg0[(size_t)r] = (int32_t)(w - beg);
            }
        }
    });
    off0[(size_t)n] = A;
    // rank = (degree, id): counting sort by degree, ids ascending inside a degree
    int32_t maxd = 0;
    for (int32_t d : deg0) maxd = d > maxd ? d : maxd;
    std::vector<int64_t> start((size_t)maxd + 2, 0);
    for (int32_t d : deg0) start[(size_t)d + 1]++;
    for (size_t d = 0; d + 1 < start.size(); ++d) start[d + 1] += start[d];
    std::vector<int32_t> rank((size_t)n), order((size_t)n);
    for (int64_t v = 0; v < n; ++v) {
        const int32_t r = (int32_t)start[(size_t)deg0[(size_t)v]]++;
        rank[(size_t)v] = r;
        order[(size_t)r] = (int32_t)v;
    }
    g.n = n;
    g.off.assign((size_t)n + 1, 0);
    for (int64_t r = 0; r < n; ++r) g.off[(size_t)r + 1] = g.off[(size_t)r] + deg0[(size_t)order[(size_t)r]];
    g.m = g.off[(size_t)n] / 2;
    g.deg.resize((size_t)n);
    g.dplus.resize((size_t)n);
    // rows by rank, sorted: the other endpoints relabelled in place (one gather each), then vertices
    // visited in rank order
    parallel_dynamic(n, 4096, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; ++v)
            for (int64_t k = off0[(size_t)v]; k < off0[(size_t)v] + deg0[(size_t)v]; ++k)
                c0[(size_t)k] = rank[(size_t)c0[(size_t)k]];
    });
    regroup_by_destination(
        n,
        [&](int64_t r) {
            const int32_t v = order[(size_t)r];
            return std::make_pair(c0.data() + off0[(size_t)v], c0.data() + off0[(size_t)v] + deg0[(size_t)v]);
        },
        [](int32_t c) { return (int64_t)c; }, n, g.off.data(), c0.data(), pairs.data(),
        [&](int64_t r0, int64_t r1) {  // degree and out-degree (entries above r) of the rows just filled
            for (int64_t r = r0; r < r1; ++r) {
                const int64_t a = g.off[(size_t)r], z = g.off[(size_t)r + 1];
                g.deg[(size_t)r] = (int32_t)(z - a);
                const int64_t split = std::upper_bound(c0.begin() + a, c0.begin() + z, (int32_t)r) - (c0.begin() + a);
                g.dplus[(size_t)r] = (int32_t)(z - a - split);
            }
        });
    buf<uint64_t>().swap(pairs);
    c0.resize((size_t)g.off[(size_t)n]);
    g.cols.swap(c0);
    g.rank.swap(rank);
    g.offp.assign((size_t)n + 1, 0);
    g.n1 = n;
    for (int64_t r = 0; r < n; ++r) {
        if (g.n1 == n && g.deg[(size_t)r] >= 2) g.n1 = r;
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

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device bytes of a triangle block: per-vertex arrays (offp, deg, dplus, queues), out-lists and t_e,
// the fallback scratch and the accumulators.
size_t tri_block_bytes(int64_t n, int64_t out_arcs, int64_t fb_scratch) {
    const int64_t nn = n > 0 ? n : 1, oa = out_arcs > 0 ? out_arcs : 1;
    return align256(8 * (size_t)(nn + 1)) + 3 * align256(4 * (size_t)nn) + align256(8 * (size_t)nn) +
           2 * align256(4 * (size_t)oa) + align256((size_t)fb_scratch) + align256(8 * (size_t)kOutLen);
}

// Device bytes of a wedge block: per-vertex arrays (off, loff, win_prefix, deg, dplus, fpos, queues,
// boundary table), sliced rows, lower lists and their reverse positions, scan scratch, accumulators.
size_t wedge_block_bytes(int64_t n, int64_t row_arcs, int64_t list_arcs) {
    const int64_t nn = n > 0 ? n : 1, ra = row_arcs > 0 ? row_arcs : 1, la = list_arcs > 0 ? list_arcs : 1;
    return 3 * align256(8 * (size_t)(nn + 1)) + 3 * align256(4 * (size_t)nn) + 2 * align256(8 * (size_t)nn) +
           align256(4 * (size_t)kGridCap * (size_t)nn) +
           align256(4 * (size_t)ra) + 2 * align256(4 * (size_t)la) + align256(8 * (size_t)kGInfo) +
           align256(8 * (scan_tmp_needed(nn) + 64)) + align256(8 * (size_t)kOutLen);
}

// Carve consecutive 256-byte aligned arrays out of one allocation.
struct Carver {
    unsigned char* p;
    template <typename T>
    T* take(size_t count) {
        T* r = reinterpret_cast<T*>(p);
        p += align256(sizeof(T) * (count > 0 ? count : 1));
        return r;
    }
};

// ------------------------------------------------------------------------------------------------
// Triangle blocks: rank ranges R, halo = out-lists of R and N+(R).
// ------------------------------------------------------------------------------------------------
struct TriBlock {
    int64_t lo, hi;
};

// Out-neighbour k of r (k < dplus[r]): the row suffix.
inline int32_t out_nbr(const RankGraph& g, int64_t r, int64_t k) {
    return g.cols[(size_t)(g.off[(size_t)r + 1] - g.dplus[(size_t)r] + k)];
}

// Exact out-arcs of the triangle halo of [lo, hi) (distinct out-lists of R and N+(R)), on all host
// cores: each vertex is claimed once through its mark byte.  mark is all zero on entry and on return.
int64_t tri_extent(const RankGraph& g, int64_t lo, int64_t hi, std::vector<uint8_t>& mark) {
    if (lo == 0 && hi == g.n) return g.offp[(size_t)g.n];  // every vertex is in the halo: all out-arcs
    std::vector<int64_t> part(host_threads(), 0);
    std::vector<std::vector<int32_t>> claimed(host_threads());
    parallel_for(hi - lo, [&](int64_t a, int64_t b, unsigned t) {
        int64_t outs = 0;
        auto add = [&](int32_t v) {  // a plain load first: hub marks are read by every thread
            if (__atomic_load_n(&mark[(size_t)v], __ATOMIC_RELAXED) == 0 &&
                __atomic_exchange_n(&mark[(size_t)v], (uint8_t)1, __ATOMIC_RELAXED) == 0) {
                claimed[t].push_back(v);
                outs += g.dplus[(size_t)v];
            }
        };
        for (int64_t u = lo + a; u < lo + b; ++u) {
            add((int32_t)u);
            for (int64_t k = 0; k < g.dplus[(size_t)u]; ++k) add(out_nbr(g, u, k));
        }
        part[t] = outs;
    });
    int64_t outs = 0;
    for (size_t t = 0; t < part.size(); ++t) {
        outs += part[t];
        for (int32_t v : claimed[t]) mark[(size_t)v] = 0;
    }
    return outs;
}

// Ranges of triangle anchors: the whole rank space when its halo fits, else one sweep that extends
// each range while its exact halo fits the budget.
harp_status cut_triangle_ranges(const RankGraph& g, uint64_t budget, int32_t parts, int64_t fb_scratch,
                                std::vector<TriBlock>& out, uint64_t& peak) {
    const int64_t n = g.n;
    std::vector<uint8_t> mark((size_t)n, 0);
    std::vector<int32_t> touched;
    auto extent = [&](int64_t lo, int64_t hi) { return tri_extent(g, lo, hi, mark); };
    if (parts == 0) {
        const int64_t all = extent(0, n);
        if (tri_block_bytes(n, all, fb_scratch) <= budget) {
            peak = std::max<uint64_t>(peak, tri_block_bytes(n, all, fb_scratch));
            out.push_back({0, n});
            return HARP_OK;
        }
    }
    if (parts > 0) {
        for (int32_t k = 0; k < parts; ++k) {
            const TriBlock b{n * k / parts, n * (k + 1) / parts};
            peak = std::max<uint64_t>(peak, tri_block_bytes(n, extent(b.lo, b.hi), fb_scratch));
            out.push_back(b);
        }
        return HARP_OK;
    }
    int64_t lo = 0;
    while (lo < n) {
        int64_t outs = 0, hi = lo;
        touched.clear();
        while (hi < n) {
            const int64_t outs0 = outs;
            const size_t t0 = touched.size();
            auto add = [&](int32_t v) {
                if (!mark[(size_t)v]) {
                    mark[(size_t)v] = 1;
                    touched.push_back(v);
                    outs += g.dplus[(size_t)v];
                }
            };
            add((int32_t)hi);
            for (int64_t k = 0; k < g.dplus[(size_t)hi]; ++k) add(out_nbr(g, hi, k));
            if (tri_block_bytes(n, outs, fb_scratch) > budget) {
                if (hi == lo) {
                    for (int32_t v : touched) mark[(size_t)v] = 0;
                    return HARP_ENOMEM;  // this vertex alone does not fit
                }
                for (size_t k = t0; k < touched.size(); ++k) mark[(size_t)touched[k]] = 0;  // undo hi
                touched.resize(t0);
                outs = outs0;
                break;
            }
            ++hi;
        }
        for (int32_t v : touched) mark[(size_t)v] = 0;
        peak = std::max<uint64_t>(peak, tri_block_bytes(n, outs, fb_scratch));
        out.push_back({lo, hi});
        lo = hi;
    }
    return HARP_OK;
}

// ------------------------------------------------------------------------------------------------
// Wedge blocks: rank ranges R of roots, each cut into x-slices X.
// ------------------------------------------------------------------------------------------------
struct WedgeBlock {
    int64_t lo, hi;    // roots
    int64_t xlo, xhi;  // opposite vertices
};

// Lower-list arcs of root u that enter a wedge block: its whole N-(u) when it can root a wedge.
int64_t list_arcs_of(const RankGraph& g, int64_t u) {
    const int64_t dm = g.deg[(size_t)u] - g.dplus[(size_t)u];
    return dm >= 2 ? dm : 0;
}

harp_status cut_wedge_blocks(const RankGraph& g, uint64_t budget, int32_t parts, std::vector<WedgeBlock>& out,
                             uint64_t& peak) {
    const int64_t n = g.n;
    std::vector<std::pair<int64_t, int64_t>> ranges;
    const size_t fixed = wedge_block_bytes(n, 0, 0);
    if (parts > 0) {
        for (int32_t k = 0; k < parts; ++k) ranges.push_back({n * k / parts, n * (k + 1) / parts});
    } else {
        // roots: their lists may take a third of what the per-vertex arrays leave
        if (fixed > budget) return HARP_ENOMEM;
        const uint64_t list_budget = (budget - fixed) / 3;
        int64_t lo = 0;
        while (lo < n) {
            int64_t hi = lo, la = 0;
            while (hi < n) {
                const int64_t add = list_arcs_of(g, hi);
                if (8 * (uint64_t)(la + add) > list_budget && hi > lo) break;
                la += add;
                ++hi;
            }
            if (8 * (uint64_t)la > list_budget) return HARP_ENOMEM;
            ranges.push_back({lo, hi});
            lo = hi;
        }
    }
    // One range over the whole graph: its rows are those of every w that is a lower neighbour of a
    // root with two or more lower neighbours, i.e. some u in N+(w) has d-(u) >= 2; each holds its
    // elements x >= n1.  Counted per w without marks; when that block fits, no slicing is needed.
    if (ranges.size() == 1 && ranges[0].first == 0 && ranges[0].second == n && n > 0) {
        std::vector<int64_t> prow(host_threads(), 0), pla(host_threads(), 0);
        parallel_for(n, [&](int64_t lo, int64_t hi, unsigned t) {
            int64_t rows = 0, la = 0;
            for (int64_t w = lo; w < hi; ++w) {
                la += list_arcs_of(g, w);
                const int64_t b = g.off[(size_t)w], e = g.off[(size_t)w + 1];
                bool lower = false;
                for (int64_t k = e - g.dplus[(size_t)w]; k < e && !lower; ++k) lower = list_arcs_of(g, g.cols[(size_t)k]) > 0;
                if (lower)
                    rows += e - (std::lower_bound(g.cols.begin() + b, g.cols.begin() + e, (int32_t)g.n1) - g.cols.begin());
            }
            prow[t] += rows;
            pla[t] += la;
        });
        int64_t rows_total = 0, la = 0;
        for (size_t t = 0; t < prow.size(); ++t) {
            rows_total += prow[t];
            la += pla[t];
        }
        if (parts > 0 || g.n1 >= n || wedge_block_bytes(n, rows_total, la) <= budget) {
            peak = std::max<uint64_t>(peak, wedge_block_bytes(n, rows_total, la));
            out.push_back({0, n, 0, n});
            return HARP_OK;
        }
    }
    // x-slices per root range, cut from a histogram of the row elements the block would hold, counted
    // per x-bucket (at most 65,536 buckets, per-thread counts, no atomics); slices end on bucket
    // boundaries, and a bucket that cannot fit alone is cut exactly, per x.
    int bs = 0;
    while ((n >> bs) >= 65536) ++bs;
    const int64_t nbk = (n >> bs) + 1;
    const unsigned nt = host_threads();
    std::vector<std::vector<int64_t>> hist(nt, std::vector<int64_t>((size_t)nbk, 0));
    std::vector<int64_t> hsum((size_t)nbk, 0);
    std::vector<std::vector<int32_t>> lower(nt);
    std::vector<int32_t> all;
    for (const auto& r : ranges) {
        const int64_t lo = r.first, hi = r.second;
        if (lo >= hi) continue;
        int64_t la = 0;
        for (int64_t u = lo; u < hi; ++u) la += list_arcs_of(g, u);
        // the block's rows are those of every w < hi with a root u in N+(w) n [lo, hi) that has two or
        // more lower neighbours; one pass over w (chunks taken dynamically: hub rows sit at the top)
        // finds them and counts their elements x in [n1, hi) per x-bucket
        for (auto& l : lower) l.clear();
        const int64_t xa = g.n1, xb = hi;  // opposite vertices of degree >= 2, below the range's end
        auto seg = [&](int32_t w, int64_t x0, int64_t x1, auto&& visit) {  // row w's elements in [x0, x1)
            const auto b = g.cols.begin() + g.off[(size_t)w], e = g.cols.begin() + g.off[(size_t)w + 1];
            for (auto it = std::lower_bound(b, e, (int32_t)x0); it != e && *it < x1; ++it) visit(*it);
        };
        {
            std::atomic<int64_t> next{0};
            std::vector<std::thread> th;
            for (unsigned t = 0; t < nt; ++t)
                th.emplace_back([&, t] {
                    std::vector<int64_t>& h = hist[t];
                    std::fill(h.begin(), h.end(), 0);
                    for (;;) {
                        const int64_t w0 = next.fetch_add(256);
                        if (w0 >= hi) break;
                        for (int64_t w = w0; w < std::min<int64_t>(w0 + 256, hi); ++w) {
                            const auto e = g.cols.begin() + g.off[(size_t)w + 1];
                            bool root = false;
                            for (auto it = std::lower_bound(g.cols.begin() + g.off[(size_t)w], e,
                                                            (int32_t)std::max<int64_t>(lo, w + 1));
                                 it != e && *it < hi && !root; ++it)
                                root = list_arcs_of(g, *it) > 0;
                            if (!root) continue;
                            lower[t].push_back((int32_t)w);
                            seg((int32_t)w, xa, xb, [&](int32_t x) { h[(size_t)(x >> bs)]++; });
                        }
                    }
                });
            for (auto& x : th) x.join();
        }
        all.clear();
        for (auto& l : lower) all.insert(all.end(), l.begin(), l.end());
        for (int64_t k = 0; k < nbk; ++k) {
            int64_t c = 0;
            for (unsigned t = 0; t < nt; ++t) c += hist[t][(size_t)k];
            hsum[(size_t)k] = c;
        }
        int64_t rows_total = 0;
        for (int64_t k = 0; k < nbk; ++k) rows_total += hsum[(size_t)k];
        if (parts > 0 || xa >= xb || wedge_block_bytes(n, rows_total, la) <= budget) {
            peak = std::max<uint64_t>(peak, wedge_block_bytes(n, rows_total, la));
            out.push_back({lo, hi, 0, n});
            continue;
        }
        int64_t x0 = xa, rows = 0;
        auto close = [&](int64_t x) {  // the slice [x0, x) holds `rows` row elements
            peak = std::max<uint64_t>(peak, wedge_block_bytes(n, rows, la));
            out.push_back({lo, hi, x0 == xa ? 0 : x0, x});
            x0 = x;
            rows = 0;
        };
        for (int64_t k = xa >> bs; k <= (xb - 1) >> bs; ++k) {
            const int64_t h = hsum[(size_t)k];
            if (wedge_block_bytes(n, rows + h, la) <= budget) {
                rows += h;
                continue;
            }
            const int64_t kb = std::max<int64_t>(k << bs, xa), ke = std::min<int64_t>((k + 1) << bs, xb);
            if (rows > 0 && wedge_block_bytes(n, h, la) <= budget) {  // close before the bucket
                close(kb);
                rows = h;
                continue;
            }
            // the bucket does not fit beside (or at all): cut it per x with exact counts
            std::vector<int64_t> px((size_t)(ke - kb), 0);
            for (int32_t w : all) seg(w, kb, ke, [&](int32_t x) { px[(size_t)(x - kb)]++; });
            for (int64_t x = kb; x < ke; ++x) {
                const int64_t c = px[(size_t)(x - kb)];
                if (wedge_block_bytes(n, rows + c, la) > budget) {
                    if (rows == 0) return HARP_ENOMEM;  // one x-value's rows alone do not fit
                    close(x);
                }
                rows += c;
            }
        }
        close(n);
    }
    return HARP_OK;
}

// Scratch the triangle kernels of a block allocate: the fallback's per-warp frontier buffers (sized
// for the largest out-degree a graph of m edges can have, sqrt(2m)) and the global-staged tier's rows
// (4096 x 4096 bits per block, one block per SM).
int64_t tri_scratch_bytes(int64_t m) {
    int64_t dmax = 1;
    while (dmax * dmax < 2 * m) ++dmax;
    const int64_t sms = num_sms();
    return sms * 8 * (dmax + 32) * 4 + (dmax > 1024 ? sms * 4096 * 128 * 4 : 0);
}

// The device results of all blocks, and where the time went.
struct PartSums {
    uint64_t T = 0, K4 = 0, C4 = 0, PAWSUM = 0;
    std::vector<uint32_t> te;  // global out-arc numbering
    double transfer_ms = 0, device_ms = 0, tri_ms = 0, wedge_ms = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // copies in | kernels | copies out | end
};

// Milliseconds between the recorded phase events of one block (after it synchronised).
void add_phase_times(PartSums& sum, bool wedge) {
    float a = 0, b = 0, c = 0;
    if (cudaEventElapsedTime(&a, sum.ev[0], sum.ev[1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, sum.ev[1], sum.ev[2]) == cudaSuccess &&
        cudaEventElapsedTime(&c, sum.ev[2], sum.ev[3]) == cudaSuccess) {
        sum.transfer_ms += a + c;
        sum.device_ms += b;
        (wedge ? sum.wedge_ms : sum.tri_ms) += b;
    }
}

harp_status check_cuda(cudaError_t e) {
    if (e == cudaSuccess) return HARP_OK;
    record_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
}

harp_status run_triangle_block(const RankGraph& g, const TriBlock& blk, int dev, int64_t fb, cudaStream_t s,
                               PartSums& sum, uint64_t& h2d, uint64_t& halo_arcs) {
    const int64_t n = g.n;
    // halo: out-lists of R and N+(R), local numbering in rank order (flags set on all host cores)
    std::vector<uint8_t> in((size_t)n, 0);
    parallel_for(blk.hi - blk.lo, [&](int64_t a, int64_t b, unsigned) {
        for (int64_t u = blk.lo + a; u < blk.lo + b; ++u) {
            __atomic_store_n(&in[(size_t)u], (uint8_t)1, __ATOMIC_RELAXED);
            for (int64_t k = 0; k < g.dplus[(size_t)u]; ++k)
                __atomic_store_n(&in[(size_t)out_nbr(g, u, k)], (uint8_t)1, __ATOMIC_RELAXED);
        }
    });
    std::vector<int64_t> offp((size_t)n + 1, 0);
    for (int64_t v = 0; v < n; ++v) offp[(size_t)v + 1] = offp[(size_t)v] + (in[(size_t)v] ? g.dplus[(size_t)v] : 0);
    const int64_t outs = offp[(size_t)n];
    buf<int32_t> colsp((size_t)(outs > 0 ? outs : 1));
    parallel_for(n, [&](int64_t lo, int64_t hi, unsigned) {
        for (int64_t v = lo; v < hi; ++v) {
            const int64_t len = offp[(size_t)v + 1] - offp[(size_t)v];
            if (len)
                std::memcpy(&colsp[(size_t)offp[(size_t)v]], &g.cols[(size_t)(g.off[(size_t)v + 1] - len)],
                            sizeof(int32_t) * (size_t)len);
        }
    });
    halo_arcs += (uint64_t)outs;
    const size_t bytes = tri_block_bytes(n, outs, fb);
    void* base = nullptr;
    HARP_TRY(check_cuda(cudaMallocAsync(&base, bytes, s)));
    Carver c{static_cast<unsigned char*>(base)};
    Workspace ws;
    ws.offp = c.take<int64_t>((size_t)n + 1);
    ws.deg = c.take<int32_t>((size_t)n);
    ws.dplus = c.take<int32_t>((size_t)n);
    ws.q_tri = c.take<int32_t>((size_t)n);
    ws.q_mid = c.take<int32_t>(2 * (size_t)n);
    ws.colsp = c.take<int32_t>((size_t)outs);
    ws.te = c.take<uint32_t>((size_t)outs);
    c.take<unsigned char>((size_t)fb);  // the triangle kernels allocate their own scratch: counted here
    ws.acc = c.take<uint64_t>(kOutLen);
    ws.own_lo = blk.lo;
    ws.own_hi = blk.hi;
    cudaEventRecord(sum.ev[0], s);
    cudaError_t e = cudaMemcpyAsync(ws.offp, offp.data(), sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && outs)
        e = cudaMemcpyAsync(ws.colsp, colsp.data(), sizeof(int32_t) * (size_t)outs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws.deg, g.deg.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.dplus, g.dplus.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.te, 0, sizeof(uint32_t) * (size_t)(outs > 0 ? outs : 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s);
    harp_status st = check_cuda(e);
    h2d += 8 * (uint64_t)(n + 1) + 4 * (uint64_t)outs + 8 * (uint64_t)n;
    harp_csr view;  // the kernels' view: global n, m and maximum degree
    view.device = dev;
    view.stream = s;
    view.n = n;
    view.m = g.m;
    view.max_deg = n ? *std::max_element(g.deg.begin(), g.deg.end()) : 0;
    harp_plan plan;
    normalise_plan(nullptr, &plan);
    cudaEventRecord(sum.ev[1], s);
    if (st == HARP_OK && n > 0) st = count_triangles_k4(&view, ws, plan, s);
    cudaEventRecord(sum.ev[2], s);
    buf<uint32_t> te_local((size_t)outs);
    uint64_t acc[kOutLen] = {0};
    if (st == HARP_OK) {
        e = cudaMemcpyAsync(acc, ws.acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && outs)
            e = cudaMemcpyAsync(te_local.data(), ws.te, sizeof(uint32_t) * (size_t)outs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(sum.ev[3], s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        st = check_cuda(e);
        if (st == HARP_OK && acc[ACC_ERR]) st = HARP_EDEVICE;
        if (st == HARP_OK) add_phase_times(sum, false);
    }
    cudaFreeAsync(base, s);
    if (st != HARP_OK) return st;
    sum.T += acc[ACC_T];
    sum.K4 += acc[ACC_K4];
    sum.PAWSUM += acc[ACC_PAWSUM];
    parallel_for(n, [&](int64_t lo, int64_t hi, unsigned) {  // local out-arcs -> global out-arc ids
        for (int64_t v = lo; v < hi; ++v) {
            const int64_t lb = offp[(size_t)v], len = offp[(size_t)v + 1] - lb, gb = g.offp[(size_t)v];
            for (int64_t k = 0; k < len; ++k) sum.te[(size_t)(gb + k)] += te_local[(size_t)(lb + k)];
        }
    });
    return HARP_OK;
}

harp_status run_wedge_block(const RankGraph& g, const WedgeBlock& blk, int dev, cudaStream_t s, PartSums& sum,
                            uint64_t& h2d, uint64_t& halo_arcs) {
    const int64_t n = g.n;
    // lower lists of the roots in R that can root a wedge
    std::vector<int64_t> loff((size_t)n + 1, 0);
    for (int64_t u = 0; u < n; ++u)
        loff[(size_t)u + 1] = loff[(size_t)u] + ((u >= blk.lo && u < blk.hi) ? list_arcs_of(g, u) : 0);
    const int64_t la = loff[(size_t)n];
    buf<int32_t> lcols((size_t)(la > 0 ? la : 1));
    std::vector<uint8_t> in((size_t)n, 0);
    parallel_for(blk.hi - blk.lo, [&](int64_t a0, int64_t b0, unsigned) {  // on all host cores
        for (int64_t u = blk.lo + a0; u < blk.lo + b0; ++u) {
            const int64_t len = loff[(size_t)u + 1] - loff[(size_t)u];
            for (int64_t a = 0; a < len; ++a) {
                const int32_t w = g.cols[(size_t)(g.off[(size_t)u] + a)];
                lcols[(size_t)(loff[(size_t)u] + a)] = w;
                __atomic_store_n(&in[(size_t)w], (uint8_t)1, __ATOMIC_RELAXED);
            }
        }
    });
    // rows of the lower neighbours, restricted to the slice [xa, xb) of opposite vertices
    const int64_t xa = std::max<int64_t>(blk.xlo, g.n1), xb = std::min<int64_t>(blk.xhi, blk.hi);
    std::vector<int64_t> off((size_t)n + 1, 0), rb((size_t)n, 0);
    parallel_for(n, [&](int64_t lo, int64_t hi, unsigned) {  // slice lengths, then a prefix sum
        for (int64_t w = lo; w < hi; ++w) {
            int64_t len = 0;
            if (in[(size_t)w] && xa < xb) {
                const auto b = g.cols.begin() + g.off[(size_t)w], e = g.cols.begin() + g.off[(size_t)w + 1];
                const auto p = std::lower_bound(b, e, (int32_t)xa);
                rb[(size_t)w] = p - g.cols.begin();
                len = std::lower_bound(p, e, (int32_t)xb) - p;
            }
            off[(size_t)w + 1] = len;
        }
    });
    for (int64_t w = 0; w < n; ++w) off[(size_t)w + 1] += off[(size_t)w];
    const int64_t ra = off[(size_t)n];
    if (la == 0 || ra == 0) return HARP_OK;  // no root or no opposite vertex: nothing to count here
    buf<int32_t> cols((size_t)ra);
    parallel_for(n, [&](int64_t lo, int64_t hi, unsigned) {
        for (int64_t w = lo; w < hi; ++w) {
            const int64_t len = off[(size_t)w + 1] - off[(size_t)w];
            if (len)
                std::memcpy(&cols[(size_t)off[(size_t)w]], &g.cols[(size_t)rb[(size_t)w]],
                            sizeof(int32_t) * (size_t)len);
        }
    });
    halo_arcs += (uint64_t)(ra + la);
    const size_t bytes = wedge_block_bytes(n, ra, la);
    void* base = nullptr;
    HARP_TRY(check_cuda(cudaMallocAsync(&base, bytes, s)));
    Carver c{static_cast<unsigned char*>(base)};
    Workspace ws;
    ws.off = c.take<int64_t>((size_t)n + 1);
    int64_t* d_loff = c.take<int64_t>((size_t)n + 1);
    ws.win_prefix = c.take<int64_t>((size_t)n + 1);
    ws.deg = c.take<int32_t>((size_t)n);
    ws.dplus = c.take<int32_t>((size_t)n);
    ws.fpos = c.take<int32_t>((size_t)n);
    ws.q_mid = c.take<int32_t>(2 * (size_t)n);
    ws.q_win = c.take<int32_t>(2 * (size_t)n);
    ws.cols = c.take<int32_t>((size_t)ra);
    int32_t* d_lcols = c.take<int32_t>((size_t)la);
    ws.rev = c.take<int32_t>((size_t)la);
    ws.ginfo = c.take<int64_t>(kGInfo);
    ws.scan_tmp_len = scan_tmp_needed(n > 0 ? n : 1) + 64;
    ws.scan_tmp = c.take<int64_t>(ws.scan_tmp_len);
    ws.acc = c.take<uint64_t>(kOutLen);
    ws.bpos = c.take<int32_t>((size_t)kGridCap * (size_t)n);
    ws.loff = d_loff;
    ws.lcols = d_lcols;
    ws.lower_arcs = la;
    ws.own_lo = blk.lo;
    ws.own_hi = blk.hi;
    ws.x_lo = xa;
    ws.x_hi = xb;
    cudaEventRecord(sum.ev[0], s);
    cudaError_t e = cudaMemcpyAsync(ws.off, off.data(), sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_loff, loff.data(), sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws.cols, cols.data(), sizeof(int32_t) * (size_t)ra, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_lcols, lcols.data(), sizeof(int32_t) * (size_t)la, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws.deg, g.deg.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.dplus, g.dplus.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.acc, 0, sizeof(uint64_t) * kOutLen, s);
    harp_status st = check_cuda(e);
    h2d += 16 * (uint64_t)(n + 1) + 4 * (uint64_t)(ra + la) + 8 * (uint64_t)n;
    harp_csr view;
    view.device = dev;
    view.stream = s;
    view.n = n;
    view.m = g.m;
    view.max_deg = 0;
    harp_plan plan;
    normalise_plan(nullptr, &plan);
    cudaEventRecord(sum.ev[1], s);
    if (st == HARP_OK) st = count_wedge_c4(&view, ws, plan, s);
    cudaEventRecord(sum.ev[2], s);
    uint64_t acc[kOutLen] = {0};
    if (st == HARP_OK) {
        e = cudaMemcpyAsync(acc, ws.acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(sum.ev[3], s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        st = check_cuda(e);
        if (st == HARP_OK && acc[ACC_ERR]) st = HARP_EDEVICE;
        if (st == HARP_OK) add_phase_times(sum, true);
    }
    cudaFreeAsync(base, s);
    if (st != HARP_OK) return st;
    sum.C4 += acc[ACC_C4];
    return HARP_OK;
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
    const auto t0 = std::chrono::steady_clock::now();
    RankGraph g;
    HARP_TRY(build_rank_graph(n, m_in, src, dst, g));
    const auto t1 = std::chrono::steady_clock::now();
    if (budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        HARP_CK(cudaMemGetInfo(&fr, &tot));
        budget_bytes = fr / 2;
    }
    const int64_t fb = tri_scratch_bytes(g.m);
    std::vector<TriBlock> tri;
    std::vector<WedgeBlock> wedge;
    uint64_t device_peak = 0, h2d = 0, halo_arcs = 0;
    HARP_TRY(cut_triangle_ranges(g, budget_bytes, parts, fb, tri, device_peak));
    HARP_TRY(cut_wedge_blocks(g, budget_bytes, parts, wedge, device_peak));
    const auto t2 = std::chrono::steady_clock::now();
    PartSums sum;
    sum.te.assign((size_t)g.offp[(size_t)n], 0);
    cudaStream_t s = nullptr;
    HARP_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    harp_status st = HARP_OK;
    for (cudaEvent_t& ev : sum.ev)
        if (st == HARP_OK) st = check_cuda(cudaEventCreate(&ev));
    for (size_t k = 0; k < tri.size() && st == HARP_OK; ++k) {
        if (tri[k].lo >= tri[k].hi || g.m == 0) continue;
        st = run_triangle_block(g, tri[k], dev, fb, s, sum, h2d, halo_arcs);
    }
    for (size_t k = 0; k < wedge.size() && st == HARP_OK; ++k) {
        if (wedge[k].lo >= wedge[k].hi || g.m == 0) continue;
        st = run_wedge_block(g, wedge[k], dev, s, sum, h2d, halo_arcs);
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    for (cudaEvent_t ev : sum.ev)
        if (ev) cudaEventDestroy(ev);
    if (st != HARP_OK) return st;
    // degree sums by owner (every vertex / edge once) and the global sum_e C(t_e, 2)
    std::vector<uint64_t> pS(host_threads(), 0), pPW(host_threads(), 0), pD(host_threads(), 0);
    parallel_for(n, [&](int64_t lo, int64_t hi, unsigned t) {
        uint64_t s3 = 0, pw = 0;
        for (int64_t r = lo; r < hi; ++r) {
            const uint64_t dr = (uint64_t)g.deg[(size_t)r];
            s3 += choose3_h(dr);
            for (int64_t k = 0; k < g.dplus[(size_t)r]; ++k)
                pw += (dr - 1) * ((uint64_t)g.deg[(size_t)out_nbr(g, r, k)] - 1);
        }
        pS[t] += s3;
        pPW[t] += pw;
    });
    parallel_for((int64_t)sum.te.size(), [&](int64_t lo, int64_t hi, unsigned t) {
        uint64_t d = 0;
        for (int64_t i = lo; i < hi; ++i) d += choose2_h(sum.te[(size_t)i]);
        pD[t] += d;
    });
    uint64_t S = 0, PW = 0, D = 0;
    for (size_t t = 0; t < pS.size(); ++t) {
        S += pS[t];
        PW += pPW[t];
        D += pD[t];
    }
    const uint64_t T = sum.T, K4 = sum.K4;
    const uint64_t P = PW - 3 * T, pawn = sum.PAWSUM - 6 * T;
    const uint64_t diamond = D - 6 * K4;
    const uint64_t c4 = sum.C4 - diamond - 3 * K4;
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
        stats->partitions = (int64_t)(tri.size() + wedge.size());
        stats->m = g.m;
        stats->halo_arcs = (int64_t)halo_arcs;
        stats->h2d_bytes = h2d;
        stats->device_peak_bytes = device_peak;
        const double total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        stats->transfer_ms = sum.transfer_ms;
        stats->device_ms = sum.device_ms;
        stats->host_ms = total - sum.transfer_ms - sum.device_ms;
        stats->graph_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        stats->cut_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
        stats->tri_ms = sum.tri_ms;
        stats->wedge_ms = sum.wedge_ms;
        stats->tri_blocks = (int64_t)tri.size();
        stats->wedge_blocks = (int64_t)wedge.size();
        stats->wedge_sliced = 0;
        for (const WedgeBlock& b : wedge) stats->wedge_sliced += (b.xlo > 0 || b.xhi < n) ? 1 : 0;
    }
    return HARP_OK;
}

extern "C" harp_status harp_partition_plan(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                                           uint64_t budget_bytes, int32_t parts, harp_partition_stats* stats,
                                           int64_t* tri_out, int64_t* wedge_out, int64_t cap) {
    if (!stats || n < 0 || m_in < 0 || (m_in > 0 && (!src || !dst)) || parts < 0 || cap < 0 ||
        (cap > 0 && (!tri_out || !wedge_out)))
        return HARP_EINVAL;
    if (n > 2147483647LL || m_in > 2147483647LL) return HARP_EOVERFLOW;
    const auto t0 = std::chrono::steady_clock::now();
    RankGraph g;
    HARP_TRY(build_rank_graph(n, m_in, src, dst, g));
    const auto t1 = std::chrono::steady_clock::now();
    if (budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        HARP_CK(cudaMemGetInfo(&fr, &tot));
        budget_bytes = fr / 2;
    }
    std::vector<TriBlock> tri;
    std::vector<WedgeBlock> wedge;
    uint64_t device_peak = 0;
    HARP_TRY(cut_triangle_ranges(g, budget_bytes, parts, tri_scratch_bytes(g.m), tri, device_peak));
    HARP_TRY(cut_wedge_blocks(g, budget_bytes, parts, wedge, device_peak));
    const auto t2 = std::chrono::steady_clock::now();
    *stats = harp_partition_stats{};
    stats->partitions = (int64_t)(tri.size() + wedge.size());
    stats->m = g.m;
    stats->device_peak_bytes = device_peak;
    stats->graph_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats->cut_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    stats->host_ms = stats->graph_ms + stats->cut_ms;
    stats->tri_blocks = (int64_t)tri.size();
    stats->wedge_blocks = (int64_t)wedge.size();
    for (const WedgeBlock& b : wedge) stats->wedge_sliced += (b.xlo > 0 || b.xhi < n) ? 1 : 0;
    for (size_t k = 0; k < tri.size() && (int64_t)k < cap; ++k) {
        tri_out[2 * k] = tri[k].lo;
        tri_out[2 * k + 1] = tri[k].hi;
    }
    for (size_t k = 0; k < wedge.size() && (int64_t)k < cap; ++k) {
        wedge_out[4 * k] = wedge[k].lo;
        wedge_out[4 * k + 1] = wedge[k].hi;
        wedge_out[4 * k + 2] = wedge[k].xlo;
        wedge_out[4 * k + 3] = wedge[k].xhi;
    }
    return HARP_OK;
}

extern "C" harp_status harp_rank_csr_host(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                                          int64_t* m_out, int32_t* rank_out, int64_t* off_out, int32_t* cols_out,
                                          int64_t cols_cap) {
    if (!m_out || n < 0 || m_in < 0 || (m_in > 0 && (!src || !dst)) || cols_cap < 0) return HARP_EINVAL;
    if (n > 2147483647LL || m_in > 2147483647LL) return HARP_EOVERFLOW;
    RankGraph g;
    HARP_TRY(build_rank_graph(n, m_in, src, dst, g));
    *m_out = g.m;
    if (rank_out) std::copy(g.rank.begin(), g.rank.end(), rank_out);
    if (off_out) std::copy(g.off.begin(), g.off.end(), off_out);
    if (cols_out && 2 * g.m <= cols_cap) std::copy(g.cols.begin(), g.cols.end(), cols_out);
    return HARP_OK;
}
