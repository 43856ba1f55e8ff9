/*
 * CPU oracle for exact connected induced 4-vertex motif counts.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or call this code; only
 * the tests, the package's smoke() check and the CPU-baseline leg of bench.py use it.  It shares no
 * source with the CUDA library.
 *
 * Count order everywhere: out[0] 3-star, out[1] 4-path, out[2] tailed triangle (paw),
 * out[3] 4-cycle, out[4] diamond, out[5] 4-clique.
 *
 * Every entry point builds its own simple undirected graph from a raw edge list (ids in [0, n);
 * self-loops dropped, duplicates merged, both directions implied).  Return value 0 = ok,
 * -1 = invalid argument (id out of range, n too large for the method), -2 = out of memory.
 */
#ifndef HARP_ORACLE_H
#define HARP_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Definition (Section II): every 4-subset S, G[S] connected, classified up to isomorphism.  n <= 512. */
int orc_count4_brute(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, uint64_t out[6]);

/* Definition, enumerated by Wernicke's ESU: each connected 4-subset is visited exactly once. */
int orc_count4_esu(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                   uint64_t out[6]);

/* The closure equations of Section III-F taken literally: per-triangle X_1, X_2, X_3; per-edge
 * A_e x B_e pair scan for paths and cycles; per-vertex H_u inclusion-exclusion for stars. */
int orc_count4_literal(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                       uint64_t out[6]);

/* Non-induced pattern counts by direct loops:
 * stats[0] T (triangles), [1] K4, [2] C4_non (4-cycles as subgraphs), [3] S_non = sum_v C(d,3),
 * [4] P_non (3-edge paths), [5] paw_non = sum_v t(v)(d_v - 2), [6] D_non = sum_e C(t_e, 2),
 * [7] m (undirected simple edges).  All sums are taken modulo 2^64. */
int orc_noninduced(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                   uint64_t stats[8]);

/* Induced counts from the non-induced counts by inverting the containment system (mod 2^64). */
void orc_induced_from_noninduced(const uint64_t stats[8], uint64_t out[6]);

/* orc_noninduced followed by orc_induced_from_noninduced. */
int orc_count4_combo(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst, int threads,
                     uint64_t out[6]);

/* Per-edge triangle counts t_e = |N(u) n N(v)| for the simple edges u < v in (u, v) lexicographic
 * order, by sorted-list merge.  eu, ev, te have room for m entries; *m_out receives m. */
int orc_edge_triangles(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                       int32_t* eu, int32_t* ev, uint32_t* te, int64_t cap, int64_t* m_out);

/* Simple-graph summary: m (undirected), max degree. */
int orc_graph_summary(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                      int64_t* m_out, int64_t* maxdeg_out);

#ifdef __cplusplus
}
#endif
#endif
