/*
 * CPU oracle for exact connected induced 4-vertex motif counts (HARP-ME, arXiv 2607.12074).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, smoke() and bench.py's CPU-baseline leg use this file;
 * the product path never does.  It shares no source, header, table or helper with the CUDA
 * library.  Everything here is plain, sequential-per-unit C; OpenMP only splits independent
 * outer loops (roots, vertices), never changes what is computed.
 *
 * Pins (what each function is checked against in tests/, besides the other functions here):
 *   orc_count4_brute    closed forms (K_n, K_{1,n}, C_n, P_n, K_{a,b}, wheels, cocktail-party,
 *                       the six motif graphs), hand-checked small examples in tests/golden/.
 *   orc_count4_esu      brute force on random tiny graphs, closed forms.
 *   orc_count4_literal  brute force / ESU; divisibility of the 1/2 and 1/4 sums.
 *   orc_noninduced      tr(A^3) = 6T and tr(A^4) = 8 C4_non + 4 sum C(d,2) + 2m by exact integer
 *                       matrix powers; the linear identities that tie the non-induced sums to the
 *                       brute-force induced counts; per-edge merge (orc_edge_triangles).
 *   orc_induced_from_noninduced  brute force on random graphs and on all closed forms.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------ */
/* The oracle's own simple-graph adjacency: rows sorted ascending, no loops, no duplicates.    */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int64_t m;      /* undirected simple edges */
    int64_t* off;   /* n + 1 */
    int32_t* adj;   /* 2m   */
} og;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void og_free(og* g) {
    free(g->off);
    free(g->adj);
    g->off = NULL;
    g->adj = NULL;
}

static int og_build(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, og* g) {
    memset(g, 0, sizeof(*g));
    if (n < 0 || n > 2147483647LL || m_in < 0) return -1;
    for (int64_t e = 0; e < m_in; ++e)
        if (src[e] < 0 || dst[e] < 0 || src[e] >= n || dst[e] >= n) return -1;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -2;
    for (int64_t e = 0; e < m_in; ++e)
        if (src[e] != dst[e]) { cnt[src[e] + 1]++; cnt[dst[e] + 1]++; }
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    int32_t* raw = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt[n] + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!raw || !fill) { free(cnt); free(raw); free(fill); return -2; }
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < m_in; ++e)
        if (src[e] != dst[e]) { raw[fill[src[e]]++] = dst[e]; raw[fill[dst[e]]++] = src[e]; }
    free(fill);
    g->n = n;
    g->off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!g->off) { free(cnt); free(raw); return -2; }
    int64_t w = 0;
    g->off[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = cnt[v], e = cnt[v + 1];
        qsort(raw + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
        for (int64_t k = b; k < e; ++k)
            if (k == b || raw[k] != raw[k - 1]) raw[w++] = raw[k];
        g->off[v + 1] = w;
    }
    free(cnt);
    g->adj = raw;
    g->m = w / 2;
    return 0;
}

static int64_t og_deg(const og* g, int64_t v) { return g->off[v + 1] - g->off[v]; }

/* is v in the sorted row of u? */
static int og_adj(const og* g, int32_t u, int32_t v) {
    int64_t lo = g->off[u], hi = g->off[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->adj[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < g->off[u + 1] && g->adj[lo] == v;
}

static int omp_threads(int threads) {
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* Binomials evaluated exactly modulo 2^64: the divisors are taken out of the factors first. */
static uint64_t choose2(uint64_t x) {
    if (x < 2) return 0;
    uint64_t a = x, b = x - 1;
    if (a % 2 == 0) a /= 2; else b /= 2;
    return a * b;
}

static uint64_t choose3(uint64_t x) {
    if (x < 3) return 0;
    uint64_t f[3] = {x, x - 1, x - 2};
    for (int i = 0; i < 3; ++i) if (f[i] % 3 == 0) { f[i] /= 3; break; }
    for (int i = 0; i < 3; ++i) if (f[i] % 2 == 0) { f[i] /= 2; break; }
    return f[0] * f[1] * f[2];
}

/* ------------------------------------------------------------------------------------------ */
/* Classification of a 4-vertex induced subgraph (Section II: G[S] isomorphic to the pattern). */
/* bits: adjacency of the pairs (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).                           */
/* Returns the motif index 0..5, or -1 if G[S] is disconnected.                                 */
/* ------------------------------------------------------------------------------------------ */
static int classify4(const int bits[6]) {
    static const int pa[6] = {0, 0, 0, 1, 1, 2};
    static const int pb[6] = {1, 2, 3, 2, 3, 3};
    int deg[4] = {0, 0, 0, 0}, parent[4] = {0, 1, 2, 3}, edges = 0;
    for (int k = 0; k < 6; ++k) {
        if (!bits[k]) continue;
        ++edges;
        deg[pa[k]]++;
        deg[pb[k]]++;
        int ra = pa[k], rb = pb[k];
        while (parent[ra] != ra) ra = parent[ra];
        while (parent[rb] != rb) rb = parent[rb];
        if (ra != rb) parent[ra] = rb;
    }
    int root = 0;
    while (parent[root] != root) root = parent[root];
    for (int v = 1; v < 4; ++v) {
        int r = v;
        while (parent[r] != r) r = parent[r];
        if (r != root) return -1;
    }
    int maxdeg = deg[0];
    for (int v = 1; v < 4; ++v) if (deg[v] > maxdeg) maxdeg = deg[v];
    switch (edges) {
        case 3: return maxdeg == 3 ? 0 : 1;   /* K_{1,3} : P_4 */
        case 4: return maxdeg == 3 ? 2 : 3;   /* paw     : C_4 */
        case 5: return 4;                     /* diamond       */
        case 6: return 5;                     /* K_4           */
        default: return -1;
    }
}

static int classify_set(const og* g, const int32_t s[4]) {
    int bits[6];
    bits[0] = og_adj(g, s[0], s[1]);
    bits[1] = og_adj(g, s[0], s[2]);
    bits[2] = og_adj(g, s[0], s[3]);
    bits[3] = og_adj(g, s[1], s[2]);
    bits[4] = og_adj(g, s[1], s[3]);
    bits[5] = og_adj(g, s[2], s[3]);
    return classify4(bits);
}

/* ------------------------------------------------------------------------------------------ */
/* Brute force over all C(n,4) subsets.                                                        */
/* ------------------------------------------------------------------------------------------ */
int orc_count4_brute(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, uint64_t out[6]) {
    if (n > 512) return -1;
    og g;
    int rc = og_build(n, m_in, src, dst, &g);
    if (rc) return rc;
    unsigned char* A = (unsigned char*)calloc((size_t)(n * n + 1), 1);
    if (!A) { og_free(&g); return -2; }
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = g.off[u]; k < g.off[u + 1]; ++k) A[u * n + g.adj[k]] = 1;
    uint64_t c[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b)
            for (int64_t cc = b + 1; cc < n; ++cc)
                for (int64_t d = cc + 1; d < n; ++d) {
                    int bits[6] = {A[a * n + b], A[a * n + cc], A[a * n + d],
                                   A[b * n + cc], A[b * n + d], A[cc * n + d]};
                    int t = classify4(bits);
                    if (t >= 0) c[t]++;
                }
    memcpy(out, c, sizeof(c));
    free(A);
    og_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* ESU (Wernicke 2006): ExtendSubgraph(V_sub, V_ext, v) with exclusive neighbourhoods.          */
/* ------------------------------------------------------------------------------------------ */
static int in_closed_nbhd(const og* g, const int32_t* sub, int ns, int32_t u) {
    for (int i = 0; i < ns; ++i)
        if (sub[i] == u || og_adj(g, sub[i], u)) return 1;
    return 0;
}

static void esu_extend(const og* g, int32_t root, int32_t* sub, int ns, const int32_t* ext, int64_t ne,
                       int32_t** stack, uint64_t c[6]) {
    if (ns == 3) {
        /* the last vertex: each w in V_ext completes one connected 4-subset */
        for (int64_t i = 0; i < ne; ++i) {
            sub[3] = ext[i];
            int t = classify_set(g, sub);
            if (t >= 0) c[t]++;
        }
        return;
    }
    int32_t* next = stack[ns];
    for (int64_t i = 0; i < ne; ++i) {
        int32_t w = ext[i];
        /* V'_ext = (V_ext minus w and the vertices already taken) + N_excl(w, V_sub) above the root */
        int64_t nn = 0;
        for (int64_t j = i + 1; j < ne; ++j) next[nn++] = ext[j];
        for (int64_t k = g->off[w]; k < g->off[w + 1]; ++k) {
            int32_t u = g->adj[k];
            if (u > root && !in_closed_nbhd(g, sub, ns, u)) next[nn++] = u;
        }
        sub[ns] = w;
        esu_extend(g, root, sub, ns + 1, next, nn, stack, c);
    }
}

int orc_count4_esu(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                   uint64_t out[6]) {
    og g;
    int rc = og_build(n, m_in, src, dst, &g);
    if (rc) return rc;
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) if (og_deg(&g, v) > maxdeg) maxdeg = og_deg(&g, v);
    uint64_t c[6] = {0, 0, 0, 0, 0, 0};
    int nt = omp_threads(threads);
    int failed = 0;
#pragma omp parallel num_threads(nt)
    {
        uint64_t lc[6] = {0, 0, 0, 0, 0, 0};
        int32_t* stack[4];
        int ok = 1;
        for (int l = 0; l < 4; ++l) {
            stack[l] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(3 * maxdeg + 4));
            if (!stack[l]) ok = 0;
        }
        if (ok) {
#pragma omp for schedule(dynamic, 16)
            for (int64_t v = 0; v < n; ++v) {
                int32_t sub[4];
                sub[0] = (int32_t)v;
                int64_t ne = 0;
                for (int64_t k = g.off[v]; k < g.off[v + 1]; ++k)
                    if (g.adj[k] > v) stack[0][ne++] = g.adj[k];
                esu_extend(&g, (int32_t)v, sub, 1, stack[0], ne, stack, lc);
            }
        } else {
#pragma omp atomic write
            failed = 1;
        }
        for (int l = 0; l < 4; ++l) free(stack[l]);
#pragma omp critical
        for (int t = 0; t < 6; ++t) c[t] += lc[t];
    }
    og_free(&g);
    if (failed) return -2;
    memcpy(out, c, sizeof(c));
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Section III-F, literally.                                                                   */
/* ------------------------------------------------------------------------------------------ */
/* |N(a) n N(b)| by merge of the sorted rows */
static int64_t common2(const og* g, int32_t a, int32_t b) {
    int64_t i = g->off[a], ie = g->off[a + 1], j = g->off[b], je = g->off[b + 1], c = 0;
    while (i < ie && j < je) {
        if (g->adj[i] < g->adj[j]) ++i;
        else if (g->adj[i] > g->adj[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

int orc_count4_literal(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                       uint64_t out[6]) {
    og g;
    int rc = og_build(n, m_in, src, dst, &g);
    if (rc) return rc;
    uint64_t X1 = 0, X2 = 0, X3 = 0, P = 0, CYC = 0, STAR = 0;
    int nt = omp_threads(threads);

    /* Triangle closure: for each triangle T = {a, b, c}, X_j(T) = # vertices outside T adjacent to
     * exactly j of a, b, c.  N_paw = sum X_1, N_diamond = sum X_2 / 2, N_clique4 = sum X_3 / 4. */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(+ : X1, X2, X3)
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t kb = g.off[a]; kb < g.off[a + 1]; ++kb) {
            int32_t b = g.adj[kb];
            if (b <= a) continue;
            for (int64_t kc = g.off[a]; kc < g.off[a + 1]; ++kc) {
                int32_t c = g.adj[kc];
                if (c <= b || !og_adj(&g, b, c)) continue;
                /* three-way merge of N(a), N(b), N(c) counting multiplicities */
                int64_t ia = g.off[a], ea = g.off[a + 1];
                int64_t ib = g.off[b], eb = g.off[b + 1];
                int64_t ic = g.off[c], ec = g.off[c + 1];
                for (;;) {
                    int32_t x = 2147483647;
                    if (ia < ea && g.adj[ia] < x) x = g.adj[ia];
                    if (ib < eb && g.adj[ib] < x) x = g.adj[ib];
                    if (ic < ec && g.adj[ic] < x) x = g.adj[ic];
                    if (x == 2147483647) break;
                    int j = 0;
                    if (ia < ea && g.adj[ia] == x) { ++j; ++ia; }
                    if (ib < eb && g.adj[ib] == x) { ++j; ++ib; }
                    if (ic < ec && g.adj[ic] == x) { ++j; ++ic; }
                    if (x == a || x == b || x == c) continue;
                    if (j == 1) ++X1;
                    else if (j == 2) ++X2;
                    else if (j == 3) ++X3;
                }
            }
        }
    }

    /* Edge closure: C_e = N(u) n N(v), A_e = N(u) \ (C_e u {v}), B_e = N(v) \ (C_e u {u});
     * pairs of A_e x B_e that are non-edges give induced 4-paths (middle edge e), edges give
     * induced 4-cycles (each cycle seen from its 4 edges). */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(+ : P, CYC)
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t kv = g.off[u]; kv < g.off[u + 1]; ++kv) {
            int32_t v = g.adj[kv];
            if (v <= u) continue;
            for (int64_t kx = g.off[u]; kx < g.off[u + 1]; ++kx) {
                int32_t x = g.adj[kx];
                if (x == v || og_adj(&g, v, x)) continue;          /* x in A_e */
                for (int64_t ky = g.off[v]; ky < g.off[v + 1]; ++ky) {
                    int32_t y = g.adj[ky];
                    if (y == (int32_t)u || og_adj(&g, (int32_t)u, y)) continue;  /* y in B_e */
                    if (og_adj(&g, x, y)) ++CYC;
                    else ++P;
                }
            }
        }
    }

    /* Star closure: with H_u = G[N(u)], the induced 3-stars centred at u number
     * C(d,3) - m(H_u)(d-2) + sum_{v in N(u)} C(deg_H(v), 2) - tau(H_u). */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(+ : STAR)
    for (int64_t u = 0; u < n; ++u) {
        uint64_t d = (uint64_t)og_deg(&g, u);
        uint64_t twice_mH = 0, sum_c2 = 0, tau = 0;
        for (int64_t kv = g.off[u]; kv < g.off[u + 1]; ++kv) {
            int32_t v = g.adj[kv];
            uint64_t dh = (uint64_t)common2(&g, (int32_t)u, v);  /* deg_H(v) */
            twice_mH += dh;
            sum_c2 += choose2(dh);
            for (int64_t kw = g.off[u]; kw < g.off[u + 1]; ++kw) {
                int32_t w = g.adj[kw];
                if (w <= v || !og_adj(&g, v, w)) continue;
                for (int64_t kx = g.off[u]; kx < g.off[u + 1]; ++kx) {
                    int32_t x = g.adj[kx];
                    if (x <= w) continue;
                    if (og_adj(&g, v, x) && og_adj(&g, w, x)) ++tau;
                }
            }
        }
        uint64_t mH = twice_mH / 2;
        uint64_t star_u = choose3(d) - mH * (d >= 2 ? d - 2 : 0) + sum_c2 - tau;
        STAR += star_u;
    }
    og_free(&g);
    if (X2 % 2 != 0 || X3 % 4 != 0 || CYC % 4 != 0) return -3;
    out[0] = STAR;
    out[1] = P;
    out[2] = X1;
    out[3] = CYC / 4;
    out[4] = X2 / 2;
    out[5] = X3 / 4;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Non-induced counts by direct loops, then the containment inversion.                         */
/* ------------------------------------------------------------------------------------------ */
/* rank(v) = (d(v), v): v is "above" u if it has larger degree, ties broken by larger id. */
static int above(const og* g, int32_t v, int32_t u) {
    int64_t dv = og_deg(g, v), du = og_deg(g, u);
    return dv > du || (dv == du && v > u);
}

int orc_noninduced(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                   uint64_t stats[8]) {
    og g;
    int rc = og_build(n, m_in, src, dst, &g);
    if (rc) return rc;
    int nt = omp_threads(threads);
    /* out-rows: N+(u) = neighbours above u, kept in id order (a subsequence of the sorted row) */
    int64_t* po = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!po) { og_free(&g); return -2; }
    po[0] = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t c = 0;
        for (int64_t k = g.off[u]; k < g.off[u + 1]; ++k) c += above(&g, g.adj[k], (int32_t)u);
        po[u + 1] = po[u] + c;
    }
    int32_t* pa = (int32_t*)malloc(sizeof(int32_t) * (size_t)(po[n] + 1));
    uint32_t* te = (uint32_t*)calloc((size_t)(po[n] + 1), sizeof(uint32_t));  /* t_e per out-arc */
    uint64_t* tv = (uint64_t*)calloc((size_t)(n + 1), sizeof(uint64_t));      /* t(v) */
    if (!pa || !te || !tv) { og_free(&g); free(po); free(pa); free(te); free(tv); return -2; }
#pragma omp parallel for num_threads(nt) schedule(static, 1024)
    for (int64_t u = 0; u < n; ++u) {
        int64_t w = po[u];
        for (int64_t k = g.off[u]; k < g.off[u + 1]; ++k)
            if (above(&g, g.adj[k], (int32_t)u)) pa[w++] = g.adj[k];
    }

    /* Triangles: each triangle {u, v, w} with u below v below w is found once, at the out-arc
     * (u, v), as w in N+(u) n N+(v); each of its three edges gets +1 in t_e, each vertex +1 in t(v). */
    uint64_t T = 0, K4 = 0;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 64) reduction(+ : T)
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t a = po[u]; a < po[u + 1]; ++a) {
            int32_t v = pa[a];
            int64_t i = po[u], ie = po[u + 1], j = po[v], je = po[v + 1];
            while (i < ie && j < je) {
                if (pa[i] < pa[j]) ++i;
                else if (pa[i] > pa[j]) ++j;
                else {
                    int32_t w = pa[i];
                    ++T;
#pragma omp atomic
                    te[a]++;
#pragma omp atomic
                    te[i]++;
#pragma omp atomic
                    te[j]++;
#pragma omp atomic
                    tv[u]++;
#pragma omp atomic
                    tv[v]++;
#pragma omp atomic
                    tv[w]++;
                    ++i;
                    ++j;
                }
            }
        }
    }

    /* 4-cliques: each K4 {u, v, w, x} in rank order is found once: at out-arc (u, v) with
     * w, x in C = N+(u) n N+(v) and x in N+(w). */
#pragma omp parallel num_threads(nt)
    {
        int64_t cap = 1;
        for (int64_t u = 0; u < n; ++u) if (po[u + 1] - po[u] > cap) cap = po[u + 1] - po[u];
        int32_t* C = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        uint64_t lk = 0;
#pragma omp for schedule(dynamic, 64)
        for (int64_t u = 0; u < n; ++u) {
            for (int64_t a = po[u]; a < po[u + 1]; ++a) {
                int32_t v = pa[a];
                int64_t i = po[u], ie = po[u + 1], j = po[v], je = po[v + 1], nc = 0;
                while (i < ie && j < je) {
                    if (pa[i] < pa[j]) ++i;
                    else if (pa[i] > pa[j]) ++j;
                    else { C[nc++] = pa[i]; ++i; ++j; }
                }
                for (int64_t s = 0; s < nc; ++s) {
                    int32_t w = C[s];
                    int64_t p = 0, q = po[w], qe = po[w + 1];
                    while (p < nc && q < qe) {
                        if (C[p] < pa[q]) ++p;
                        else if (C[p] > pa[q]) ++q;
                        else { ++lk; ++p; ++q; }
                    }
                }
            }
        }
        free(C);
#pragma omp atomic
        K4 += lk;
    }

    /* 4-cycles as subgraphs (Chiba-Nishizeki): u = the top-ranked vertex of the cycle, x the
     * opposite corner; cnt[x] = # w adjacent to both with w and x below u.  Each cycle is one
     * pair {w1, w2} at exactly one (u, x). */
    uint64_t C4 = 0;
#pragma omp parallel num_threads(nt)
    {
        uint32_t* cnt = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
        int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
        uint64_t lc = 0;
#pragma omp for schedule(dynamic, 64)
        for (int64_t u = 0; u < n; ++u) {
            int64_t nt2 = 0;
            for (int64_t k = g.off[u]; k < g.off[u + 1]; ++k) {
                int32_t w = g.adj[k];
                if (!above(&g, (int32_t)u, w)) continue;
                for (int64_t k2 = g.off[w]; k2 < g.off[w + 1]; ++k2) {
                    int32_t x = g.adj[k2];
                    if (!above(&g, (int32_t)u, x)) continue;
                    if (cnt[x]++ == 0) touched[nt2++] = x;
                }
            }
            for (int64_t s = 0; s < nt2; ++s) {
                lc += choose2(cnt[touched[s]]);
                cnt[touched[s]] = 0;
            }
        }
        free(cnt);
        free(touched);
#pragma omp atomic
        C4 += lc;
    }

    /* degree and per-edge sums */
    uint64_t S = 0, Pw = 0, paw = 0, D = 0;
#pragma omp parallel for num_threads(nt) schedule(static, 1024) reduction(+ : S, Pw, paw, D)
    for (int64_t u = 0; u < n; ++u) {
        uint64_t du = (uint64_t)og_deg(&g, u);
        S += choose3(du);
        paw += tv[u] * (du >= 2 ? du - 2 : 0);
        for (int64_t a = po[u]; a < po[u + 1]; ++a) {
            uint64_t dv = (uint64_t)og_deg(&g, pa[a]);
            Pw += (du - 1) * (dv - 1);
            D += choose2(te[a]);
        }
    }
    stats[0] = T;
    stats[1] = K4;
    stats[2] = C4;
    stats[3] = S;
    stats[4] = Pw - 3 * T;
    stats[5] = paw;
    stats[6] = D;
    stats[7] = (uint64_t)g.m;
    og_free(&g);
    free(po);
    free(pa);
    free(te);
    free(tv);
    return 0;
}

/* Copies of each non-induced pattern inside each induced class (rows: non-induced pattern,
 * columns: star, path, paw, C4, diamond, K4):
 *   S_non   = star + paw + 2 diamond + 4 K4                 (a vertex with 3 chosen neighbours)
 *   P_non   = path + 2 paw + 4 C4 + 6 diamond + 12 K4       (3-edge paths)
 *   paw_non = paw + 4 diamond + 12 K4                       (triangle + pendant edge)
 *   C4_non  = C4 + diamond + 3 K4                           (4-cycles)
 *   D_non   = diamond + 6 K4                                (two triangles sharing an edge)
 *   K4      = K4
 * The system is unit upper-triangular, so back-substitution is exact modulo 2^64. */
void orc_induced_from_noninduced(const uint64_t s[8], uint64_t out[6]) {
    uint64_t k4 = s[1];
    uint64_t diamond = s[6] - 6 * k4;
    uint64_t c4 = s[2] - diamond - 3 * k4;
    uint64_t paw = s[5] - 4 * diamond - 12 * k4;
    uint64_t path = s[4] - 2 * paw - 4 * c4 - 6 * diamond - 12 * k4;
    uint64_t star = s[3] - paw - 2 * diamond - 4 * k4;
    out[0] = star;
    out[1] = path;
    out[2] = paw;
    out[3] = c4;
    out[4] = diamond;
    out[5] = k4;
}

int orc_count4_combo(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                     uint64_t out[6]) {
    uint64_t s[8];
    int rc = orc_noninduced(n, m_in, src, dst, threads, s);
    if (rc) return rc;
    orc_induced_from_noninduced(s, out);
    return 0;
}

int orc_edge_triangles(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                       int32_t* eu, int32_t* ev, uint32_t* te, int64_t cap, int64_t* m_out) {
    og g;
    int rc = og_build(n, m_in, src, dst, &g);
    if (rc) return rc;
    *m_out = g.m;
    if (g.m > cap) { og_free(&g); return -1; }
    int64_t e = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = g.off[u]; k < g.off[u + 1]; ++k) {
            int32_t v = g.adj[k];
            if (v <= u) continue;
            eu[e] = (int32_t)u;
            ev[e] = v;
            te[e] = (uint32_t)common2(&g, (int32_t)u, v);
            ++e;
        }
    og_free(&g);
    return 0;
}

int orc_graph_summary(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                      int64_t* m_out, int64_t* maxdeg_out) {
    og g;
    int rc = og_build(n, m_in, src, dst, &g);
    if (rc) return rc;
    int64_t md = 0;
    for (int64_t v = 0; v < n; ++v) if (og_deg(&g, v) > md) md = og_deg(&g, v);
    *m_out = g.m;
    *maxdeg_out = md;
    og_free(&g);
    return 0;
}
