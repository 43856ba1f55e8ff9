/*
 * Seeded synthetic graph generators (edge lists only).
 *
 * This module produces the inputs that both the CPU oracle and the GPU path
 * consume.  It holds none of the motif-counting arithmetic: it only draws
 * random undirected edge lists.  Output lists may contain duplicates and
 * self-loops (R-MAT, Chung-Lu); both consumers drop them when they build
 * their own adjacency structures.
 *
 * Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), written out here so that the
 * same seed gives the same graph on x86-64 and on AArch64.  No <random>
 * distributions and no libm calls decide an edge except sqrt/log/pow in the
 * RGG and Chung-Lu weights, whose inputs are exactly representable doubles.
 *
 * Generators (graph families of the paper's evaluation, Section IV-B):
 *   - Barabasi-Albert preferential attachment (social-like skew),
 *   - Erdos-Renyi G(n, p) by geometric skipping (Batagelj-Brandes 2005),
 *   - random geometric graph in the unit square (localised, bio-like),
 *   - R-MAT recursive matrix (Chakrabarti, Zhan, Faloutsos 2004),
 *   - Chung-Lu expected-degree power law (Miller-Hagberg 2011 skipping).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s; } gg_rng;

static uint64_t gg_next(gg_rng* r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* A stream is identified by (seed, purpose); streams do not overlap in practice. */
static gg_rng gg_stream(uint64_t seed, uint64_t purpose) {
    gg_rng r;
    r.s = seed * 0xD1B54A32D192ED03ULL + purpose * 0x8CB92BA72F3D8DD7ULL + 0x2545F4914F6CDD1DULL;
    gg_next(&r);
    return r;
}

/* uniform double in [0, 1) with 53 random bits */
static double gg_unif(gg_rng* r) { return (double)(gg_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, k) by 128-bit multiply-shift (Lemire 2019; bias < k / 2^64) */
static uint64_t gg_below(gg_rng* r, uint64_t k) {
    return (uint64_t)(((unsigned __int128)gg_next(r) * (unsigned __int128)k) >> 64);
}

uint64_t gg_splitmix64_at(uint64_t seed, uint64_t purpose, int64_t index) {
    gg_rng r = gg_stream(seed, purpose);
    uint64_t v = 0;
    for (int64_t i = 0; i <= index; ++i) v = gg_next(&r);
    return v;
}

/* ---------------------------------------------------------------------------
 * Barabasi-Albert: seed graph K_{m+1} on vertices 0..m, then every new vertex
 * attaches to m distinct existing vertices chosen with probability
 * proportional to degree (uniform draw from the list of edge endpoints,
 * duplicates redrawn).  Edge count = C(m+1,2) + (n-m-1)*m for n > m.
 * Returns the number of edges written (cap must be >= that), or -1.
 * ------------------------------------------------------------------------- */
int64_t gg_ba(int64_t n, int32_t m, uint64_t seed, int32_t* src, int32_t* dst, int64_t cap) {
    if (n <= 0 || m <= 0) return 0;
    int64_t k0 = (n < (int64_t)m + 1) ? n : (int64_t)m + 1;
    int64_t need = k0 * (k0 - 1) / 2 + (n > k0 ? (n - k0) * (int64_t)m : 0);
    if (need > cap) return -1;
    gg_rng r = gg_stream(seed, 1);
    int32_t* ends = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * need + 1));
    if (!ends) return -1;
    int64_t ne = 0, e = 0;
    for (int64_t a = 0; a < k0; ++a)
        for (int64_t b = a + 1; b < k0; ++b) {
            src[e] = (int32_t)a; dst[e] = (int32_t)b; ++e;
            ends[ne++] = (int32_t)a; ends[ne++] = (int32_t)b;
        }
    int32_t* pick = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    for (int64_t v = k0; v < n; ++v) {
        int got = 0;
        while (got < m) {
            int32_t t = ends[gg_below(&r, (uint64_t)ne)];
            int dup = 0;
            for (int i = 0; i < got; ++i) if (pick[i] == t) { dup = 1; break; }
            if (!dup) pick[got++] = t;
        }
        for (int i = 0; i < m; ++i) {
            src[e] = (int32_t)v; dst[e] = pick[i]; ++e;
            ends[ne++] = (int32_t)v; ends[ne++] = pick[i];
        }
    }
    free(pick);
    free(ends);
    return e;
}

/* ---------------------------------------------------------------------------
 * Erdos-Renyi G(n, p) by geometric skipping over the pairs (v, w), w < v.
 * Returns the edge count, or -(needed) if cap is too small (caller retries).
 * ------------------------------------------------------------------------- */
int64_t gg_er(int64_t n, double p, uint64_t seed, int32_t* src, int32_t* dst, int64_t cap) {
    if (n <= 1 || p <= 0.0) return 0;
    gg_rng r = gg_stream(seed, 2);
    int64_t e = 0, over = 0;
    if (p >= 1.0) {
        for (int64_t v = 1; v < n; ++v)
            for (int64_t w = 0; w < v; ++w) {
                if (e < cap) { src[e] = (int32_t)v; dst[e] = (int32_t)w; } else over = 1;
                ++e;
            }
        return over ? -e : e;
    }
    double lq = log(1.0 - p);
    int64_t v = 1, w = -1;
    while (v < n) {
        double u = 1.0 - gg_unif(&r);          /* in (0, 1] */
        w = w + 1 + (int64_t)floor(log(u) / lq);
        while (w >= v && v < n) { w -= v; ++v; }
        if (v < n) {
            if (e < cap) { src[e] = (int32_t)v; dst[e] = (int32_t)w; } else over = 1;
            ++e;
        }
    }
    return over ? -e : e;
}

/* ---------------------------------------------------------------------------
 * Random geometric graph: n points uniform in the unit square (no torus),
 * edge iff Euclidean distance < radius.  Cell grid of side >= radius.
 * Returns the edge count or -(needed).
 * ------------------------------------------------------------------------- */
int64_t gg_rgg(int64_t n, double radius, uint64_t seed, int32_t* src, int32_t* dst, int64_t cap) {
    if (n <= 1 || radius <= 0.0) return 0;
    gg_rng r = gg_stream(seed, 3);
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { x[i] = gg_unif(&r); y[i] = gg_unif(&r); }
    int64_t g = (int64_t)floor(1.0 / radius);
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    int64_t ncell = g * g;
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    memset(head, 0, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = (int64_t)(x[i] * (double)g); if (cx >= g) cx = g - 1;
        int64_t cy = (int64_t)(y[i] * (double)g); if (cy >= g) cy = g - 1;
        cell[i] = cx * g + cy;
        head[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c + 1] += head[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, head, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = i;  /* ascending i within a cell */
    double r2 = radius * radius;
    int64_t e = 0, over = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = cell[i] / g, cy = cell[i] % g;
        for (int64_t dx = -1; dx <= 1; ++dx)
            for (int64_t dy = -1; dy <= 1; ++dy) {
                int64_t ax = cx + dx, ay = cy + dy;
                if (ax < 0 || ay < 0 || ax >= g || ay >= g) continue;
                int64_t c = ax * g + ay;
                for (int64_t k = head[c]; k < head[c + 1]; ++k) {
                    int64_t j = order[k];
                    if (j <= i) continue;
                    double ddx = x[i] - x[j], ddy = y[i] - y[j];
                    if (ddx * ddx + ddy * ddy < r2) {
                        if (e < cap) { src[e] = (int32_t)i; dst[e] = (int32_t)j; } else over = 1;
                        ++e;
                    }
                }
            }
    }
    free(x); free(y); free(head); free(order); free(cell); free(fill);
    return over ? -e : e;
}

/* ---------------------------------------------------------------------------
 * R-MAT: ef * 2^scale directed draws; at each of `scale` levels the quadrant
 * is a, b, c, d with the given probabilities (row bit set for c, d; column
 * bit set for b, d).  No noise.  Vertex ids are then relabelled by a seeded
 * Fisher-Yates permutation so that id order carries no degree information.
 * Self-loops and duplicate pairs are kept (consumers drop them).
 * ------------------------------------------------------------------------- */
int64_t gg_rmat(int32_t scale, int64_t ef, double a, double b, double c, uint64_t seed,
                int32_t* src, int32_t* dst, int64_t cap) {
    if (scale <= 0 || scale > 30) return 0;
    int64_t n = (int64_t)1 << scale;
    int64_t M = ef * n;
    if (M > cap) return -M;
    gg_rng r = gg_stream(seed, 4);
    double ab = a + b, abc = a + b + c;
    for (int64_t e = 0; e < M; ++e) {
        int64_t i = 0, j = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double q = gg_unif(&r);
            int64_t bi = (q >= ab) ? 1 : 0;
            int64_t bj = ((q >= a && q < ab) || q >= abc) ? 1 : 0;
            i |= bi << l; j |= bj << l;
        }
        src[e] = (int32_t)i; dst[e] = (int32_t)j;
    }
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    gg_rng rp = gg_stream(seed, 5);
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t k = (int64_t)gg_below(&rp, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[k]; perm[k] = t;
    }
    for (int64_t e = 0; e < M; ++e) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
    free(perm);
    return M;
}

/* ---------------------------------------------------------------------------
 * Chung-Lu: vertex weights w_i = c * (i + i0)^(-1/(gamma-1)), i = 0..n-1,
 * sorted non-increasing; pair (i, j), i < j, is an edge with probability
 * min(1, w_i w_j / S), S = sum w.  Sampled by the Miller-Hagberg skipping
 * method (each row i scans j > i with a geometric skip under the current
 * upper bound p = min(1, w_i w_j / S), then accepts with q / p).
 * Returns the edge count or -(needed) if cap is too small.
 * ------------------------------------------------------------------------- */
/* The expected-degree weights w_i = c (i + i0)^(-1/(gamma-1)) and their sum S (in index order). */
static double cl_weights(int64_t n, double gamma, double c, double i0, double* w) {
    double ex = -1.0 / (gamma - 1.0);
    double S = 0.0;
    for (int64_t i = 0; i < n; ++i) { w[i] = c * pow((double)i + i0, ex); S += w[i]; }
    return S;
}

/* Row u of the Miller-Hagberg process: every pair (u, v), v > u, is an edge with probability
 * min(1, w_u w_v / S), drawn from row u's own stream.  emit(v) is called for each edge. */
#define CL_ROW(u, ...)                                                         \
    do {                                                                       \
        gg_rng r_ = gg_stream(seed, 0x100000000ULL + (uint64_t)(u));           \
        int64_t v = (u) + 1;                                                   \
        double p_ = w[u] * w[v < n ? v : n - 1] / S;                           \
        if (p_ > 1.0) p_ = 1.0;                                                \
        while (v < n && p_ > 0.0) {                                            \
            if (p_ < 1.0) {                                                    \
                double q_ = 1.0 - gg_unif(&r_);                                \
                v += (int64_t)floor(log(q_) / log(1.0 - p_));                  \
            }                                                                  \
            if (v < n) {                                                       \
                double qq_ = w[u] * w[v] / S;                                  \
                if (qq_ > 1.0) qq_ = 1.0;                                      \
                if (gg_unif(&r_) < qq_ / p_) { __VA_ARGS__; }                  \
                p_ = qq_;                                                      \
                ++v;                                                           \
            }                                                                  \
        }                                                                      \
    } while (0)

int64_t gg_chung_lu(int64_t n, double gamma, double c, double i0, uint64_t seed,
                    int64_t row_lo, int64_t row_hi,
                    int32_t* src, int32_t* dst, int64_t cap) {
    if (n <= 1) return 0;
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double S = cl_weights(n, gamma, c, i0, w);
    int64_t e = 0, over = 0;
    if (row_hi > n) row_hi = n;
    for (int64_t u = row_lo; u < row_hi; ++u) {
        CL_ROW(u, {
            if (e < cap) { src[e] = (int32_t)u; dst[e] = (int32_t)v; } else over = 1;
            ++e;
        });
    }
    free(w);
    return over ? -e : e;
}

/* The subgraph of gg_chung_lu(n, ...) induced on the vertex set sub[0 .. k) (sorted, distinct), its
 * vertices renumbered by their index in sub.  Rows are independent streams, so only the rows of sub
 * are drawn: the edges of row u = sub[i] whose other end lies in sub, for i in [i_lo, i_hi). */
int64_t gg_chung_lu_induced(int64_t n, double gamma, double c, double i0, uint64_t seed,
                            const int32_t* sub, int64_t k, int64_t i_lo, int64_t i_hi,
                            int32_t* src, int32_t* dst, int64_t cap) {
    if (n <= 1 || k <= 0) return 0;
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double S = cl_weights(n, gamma, c, i0, w);
    int64_t e = 0, over = 0;
    if (i_hi > k) i_hi = k;
    for (int64_t i = i_lo; i < i_hi; ++i) {
        const int64_t u = sub[i];
        CL_ROW(u, {
            int64_t lo = i + 1, hi = k; /* v > u: its index, if any, lies after i */
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if ((int64_t)sub[mid] < v) lo = mid + 1; else hi = mid;
            }
            if (lo < k && (int64_t)sub[lo] == v) {
                if (e < cap) { src[e] = (int32_t)i; dst[e] = (int32_t)lo; } else over = 1;
                ++e;
            }
        });
    }
    free(w);
    return over ? -e : e;
}
