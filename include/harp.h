/*
 * harp.h - C ABI of libharp: exact connected induced 4-vertex motif counts on one GB300 (sm_103a).
 *
 * Method: HARP-ME (Kumar, Nasre; arXiv 2607.12074).  An anchor basis is enumerated explicitly over a
 * degree-ordered CSR (Section III-A/B: triangles with per-edge triangle statistics, their 4-clique
 * extensions, and ordered wedges), driven by sorted-adjacency set intersections (Section III-D), and
 * the six induced counts follow from exact closure relations (Section III-F).
 *
 * Counts (uint64, exact; arithmetic is modulo 2^64 and every result is exact whenever the true
 * count is below 2^64) are always reported in this order:
 *   [0] 3-star  [1] 4-path  [2] tailed triangle (paw)  [3] 4-cycle  [4] diamond  [5] 4-clique
 * An occurrence is a 4-vertex subset S whose induced subgraph G[S] is connected and isomorphic to the
 * motif (Section II); subsets are counted, not embeddings.
 *
 * Conventions for every entry point:
 *   - No exceptions cross this boundary; every call returns a harp_status.
 *   - Output arguments are written only when the call returns HARP_OK.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Graphs are simple and undirected.  Input edge lists may list an edge once or twice, may hold
 *     duplicates and self-loops; duplicates and self-loops are dropped.  Vertex ids are int32 in
 *     [0, n), n <= 2^31 - 1.  Any id outside [0, n) makes the call fail with HARP_EINVAL.
 *   - Device memory owned by the library is allocated with the stream-ordered allocator on the
 *     current device; handles are tied to the device that was current when they were created.
 */
#ifndef HARP_H
#define HARP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HARP_ABI_VERSION 2u  /* plans of version 1 (without the cache fields) are still accepted */

typedef enum harp_status {
    HARP_OK = 0,
    HARP_EINVAL = 1,     /* bad argument: NULL pointer, negative size, vertex id out of range      */
    HARP_ENOMEM = 2,     /* device or host allocation failed, or a request exceeds a memory budget */
    HARP_ECUDA = 3,      /* a CUDA runtime call failed; harp_last_cuda_error() gives the code      */
    HARP_EOVERFLOW = 4,  /* a size does not fit the index types (e.g. more than 2^31-1 vertices)   */
    HARP_EAGAIN = 5,     /* not finished yet / queue full: call again                               */
    HARP_ETIMEOUT = 6,   /* a bounded device-side wait ran out; the context stays usable            */
    HARP_ENOTFOUND = 7,  /* unknown ticket or handle                                                */
    HARP_EDEVICE = 8     /* a device-side consistency check failed (the kernel skipped the access)  */
} harp_status;

/* where the pointers passed to harp_build_csr live */
#define HARP_PTR_HOST 0u
#define HARP_PTR_DEVICE 1u

enum {
    HARP_STAR3 = 0, HARP_PATH4 = 1, HARP_PAW = 2, HARP_CYCLE4 = 3, HARP_DIAMOND = 4, HARP_CLIQUE4 = 5
};

/* Intermediate anchor statistics (non-induced pattern counts, modulo 2^64), as reported by
 * harp_count4_stats.  The closure of Section III-F maps these to the six induced counts. */
enum {
    HARP_STAT_TRIANGLES = 0,   /* T = number of triangles                                     */
    HARP_STAT_K4 = 1,          /* 4-cliques                                                    */
    HARP_STAT_C4 = 2,          /* 4-cycles as (not necessarily induced) subgraphs              */
    HARP_STAT_STARS = 3,       /* sum_v C(d_v, 3)                                              */
    HARP_STAT_PATHS = 4,       /* 3-edge paths: sum_e (d_u - 1)(d_v - 1) - 3T                  */
    HARP_STAT_PAWS = 5,        /* triangle + pendant edge: sum over triangles (sum of d - 6)   */
    HARP_STAT_DIAMONDS = 6,    /* two triangles sharing an edge: sum_e C(t_e, 2)               */
    HARP_STAT_EDGES = 7,       /* m, undirected simple edges                                   */
    HARP_NSTATS = 8
};

/* ------------------------------------------------------------------------------------------------
 * Graph handle (Section II: G = (V, E) simple undirected; Section III-D: sorted CSR adjacency).
 * ---------------------------------------------------------------------------------------------- */
typedef struct harp_csr harp_csr;

/* Build a device-resident symmetric CSR (int64 offsets[n+1], int32 cols[2m], every row sorted
 * ascending, no self-loops, no duplicates) from an undirected edge list of m_in pairs.
 *   n        number of vertices (ids [0, n)); 0 <= n <= 2^31 - 1
 *   m_in     number of input pairs (src[i], dst[i]); 0 <= m_in <= 2^31 - 1
 *   src,dst  int32[m_in]; host memory if flags == HARP_PTR_HOST, device memory if HARP_PTR_DEVICE.
 *            Read only; the caller keeps ownership.  Host arrays are copied in on `stream`.
 *   stream   cudaStream_t (as void*) for all work of this call; the call returns after the stream
 *            has finished it (it reads the deduplicated edge count back to size the result).
 *   out      receives a new handle owning its device memory; free it with harp_csr_free.
 * Errors: HARP_EINVAL (NULL pointers with m_in > 0, negative sizes, an id outside [0, n)),
 * HARP_EOVERFLOW (n or m_in above 2^31 - 1), HARP_ENOMEM, HARP_ECUDA. */
harp_status harp_build_csr(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                           uint32_t flags, void* stream, harp_csr** out);

/* Release a handle and all device memory it owns (stream-ordered on the handle's stream; returns
 * without waiting for the frees).
 * NULL is accepted and ignored. */
void harp_csr_free(harp_csr* g);

/* Summary of a handle: n, m (undirected simple edges), maximum degree, device bytes held (CSR plus
 * cached counting workspace).  Any output pointer may be NULL. */
harp_status harp_csr_info(const harp_csr* g, int64_t* n, int64_t* m_undirected, int64_t* max_degree,
                          size_t* device_bytes);

/* Device pointers of the CSR arrays (owned by the handle, valid until harp_csr_free):
 * offsets int64[n+1], cols int32[2m]. */
harp_status harp_csr_arrays(const harp_csr* g, const int64_t** offsets, const int32_t** cols);

/* ------------------------------------------------------------------------------------------------
 * Anchor plan (Section III-A, Eq. 1; Section III-B).  A plan chooses which exact anchor basis is
 * enumerated and how (intersection variant, warp-local vs CTA thresholds, cache sizes).  A plan
 * never changes the counts, only the work.  All-zero fields mean "library default".
 * ---------------------------------------------------------------------------------------------- */
#define HARP_BASIS_TRIANGLE_WEDGE 0u  /* triangles + per-edge t_e + 4-clique extension + wedges  */
/* The closure equations of Section III-F executed as printed: per triangle T the counts X_1, X_2, X_3
 * of outside vertices adjacent to exactly 1, 2, 3 of T (paw = sum X_1, diamond = sum X_2 / 2,
 * 4-clique = sum X_3 / 4); per edge e = (u, v) the pairs of A_e x B_e (4-path = non-edges, 4-cycle =
 * edges / 4); per vertex u the star form on H_u = G[N(u)].  The 2-vertex frontiers it reads (common
 * neighbours of an edge; of a non-adjacent pair) go through the signature cache of Section III-C,
 * keyed by the generating pair and its adjacency / non-adjacency mask.  Same counts as the
 * triangle-wedge basis, far more work on skewed graphs (harp_select_anchors weighs the two by Eq. 1).
 * Single graphs only (harp_count4, harp_count4_stats, harp_count4_async). */
#define HARP_BASIS_LITERAL 1u

/* Frontier membership probes.  With HARP_PROBE_HASH a CTA-mode anchor whose N+(u) spans few ranks
 * uses a direct table indexed by the rank offset from min N+(u) instead of the hash (exact either way). */
#define HARP_PROBE_HASH 1u     /* frontier membership by a shared-memory hash of N+(u)             */
#define HARP_PROBE_BSEARCH 2u  /* frontier membership by binary search in the sorted N+(u)         */

#define HARP_PLAN_NO_GRAPH 1u  /* flags: launch kernels one by one instead of a captured CUDA graph */
#define HARP_PLAN_NO_REUSE 2u  /* flags: signature reuse off: every 4-clique extension recomputes  */
                               /* |N+(w) n S_uv| from N+(w) instead of reading the staged frontier */
                               /* of (u, w) (Section III-C); the literal basis computes every      */
                               /* frontier instead of reading the signature cache; the counts are  */
                               /* identical                                                        */
#define HARP_PLAN_NO_BAND_MERGE 4u /* flags: keep every wedge counter width (3, 4, 5, 6, 8, 16, 32  */
                                   /* bits by the degree of x) as its own band of windows instead of */
                                   /* merging narrow bands that would cost more windows; the counts  */
                                   /* are identical                                                  */

typedef struct harp_plan {
    uint32_t version;            /* HARP_ABI_VERSION                                               */
    uint32_t basis;              /* HARP_BASIS_*                                                   */
    uint32_t tri_probe;          /* HARP_PROBE_* for the triangle / 4-clique anchor                */
    uint32_t tri_warp_max;       /* out-degree <= this (<= 32): warp-local mode; above: CTA mode   */
    uint32_t tri_cta_max;        /* out-degree <= this (<= 1024): frontiers staged in shared memory */
                                 /* (CTA mode)                                                      */
    uint32_t tri_big_max;        /* out-degree <= this (<= 4096), above tri_cta_max: frontiers      */
                                 /* staged in an L2-resident global scratch; above: unstaged        */
                                 /* fallback, every extension a miss                                */
    uint32_t c4_warp_max_work;   /* wedge work W(u) <= this: warp-local hash table                 */
    uint32_t c4_cta_max_work;    /* W(u) <= this (at most 2048): the middle tier, a warp-local hash */
                                 /* table of 4096 slots; above: windowed counters (<= c4_warp_max_ */
                                 /* work turns the middle tier off)                                */
    uint32_t c4_window_bytes;    /* shared-memory bytes of one dense counter window: 200, 100, 64   */
                                 /* or 48 KiB (the largest that fits); 0 = by graph: 200 KiB for a */
                                 /* single graph of more than 2^22 vertices, else 100 KiB          */
    uint32_t flags;              /* HARP_PLAN_*                                                    */
    /* Eq. 1 terms estimated from a sample of the graph (filled by harp_select_anchors) */
    double est_enum;             /* explicit anchor-enumeration work (wedges + 2-paths)            */
    double est_inter;            /* set-intersection probes                                        */
    double est_halo;             /* halo replication under the current memory budget (1 = none)    */
    double est_reuse;            /* fraction of frontier reads expected to repeat (reuse)          */
    double est_yield;            /* closure yield: induced counts recoverable from the statistics */
    double objective;            /* value of the Eq. 1 objective for the chosen basis              */
    /* version >= 2 only (a version-1 plan ends at `objective` and gets the defaults below) */
    uint32_t lit_cache_log2;     /* literal basis: signature-cache slots = 2^this (0 = sized from m, */
                                 /* at most 2^25; 16 bytes a slot)                                  */
    uint32_t lit_cache_min_deg;  /* literal basis: degree bin admitted to the cache: a frontier is   */
                                 /* cached only if both generating vertices have degree >= this     */
                                 /* (smaller ones are recomputed; 0 = all)                          */
    uint8_t tri_probe_bin[4];    /* HARP_PROBE_* per triangle degree bin, 0 = tri_probe: [0] warp-local */
                                 /* (out-degree <= tri_warp_max), [1] CTA <= 256, [2] CTA <= 512,    */
                                 /* [3] CTA <= 1024 (the global-staged and fallback modes always     */
                                 /* binary-search)                                                   */
    uint32_t reserved0;          /* 0                                                               */
    double est_cost_tw;          /* Eq. 1 objective of the triangle-wedge basis (harp_select_anchors) */
    double est_cost_lit;         /* Eq. 1 objective of the literal basis                          */
} harp_plan;

typedef struct harp_select_opts {
    uint64_t sample_vertices;    /* vertices sampled for the estimates (0 = 4096)                  */
    uint64_t seed;               /* sampling seed                                                  */
    uint64_t memory_budget;      /* bytes; 0 = free device memory.  Feeds the halo term.           */
    double lambda_inter, lambda_halo, lambda_reuse, lambda_yield;  /* 0 = normalised defaults     */
} harp_select_opts;

/* Fill *out with the plan chosen by the Eq. 1 objective for this graph: both legal bases
 * (HARP_BASIS_TRIANGLE_WEDGE, HARP_BASIS_LITERAL) are scored from a sample of arcs (degrees and the
 * exact common-neighbour count of each sampled arc) and the cheaper one is chosen; est_cost_tw and
 * est_cost_lit hold both objectives.  opts may be NULL. */
harp_status harp_select_anchors(const harp_csr* g, const harp_select_opts* opts, harp_plan* out);

/* ------------------------------------------------------------------------------------------------
 * Counting (the hot path).
 * ---------------------------------------------------------------------------------------------- */

/* Count the six induced motifs of g.  plan may be NULL (library default plan).  Runs on the
 * handle's stream and returns after the counts are on the host in counts_out[6]. */
harp_status harp_count4(const harp_csr* g, const harp_plan* plan, uint64_t counts_out[6]);

/* Signature-reuse counters of the last blocking count on g (harp_count4 / harp_count4_stats)
 * (Section III-C).  Triangle-wedge basis: lookups = 4-clique extensions (one per triangle), hits =
 * those answered by a staged frontier.  Literal basis: lookups = frontier requests to the signature
 * cache (common neighbours of an edge or of a non-adjacent pair), hits = those found in it.
 * HARP_ENOTFOUND before the first blocking count. */
harp_status harp_reuse_stats(const harp_csr* g, uint64_t* lookups, uint64_t* hits);

/* As harp_count4, and also return the anchor statistics (HARP_STAT_* order) in stats_out[8]. */
harp_status harp_count4_stats(const harp_csr* g, const harp_plan* plan, uint64_t counts_out[6],
                              uint64_t stats_out[8]);

/* Asynchronous form: enqueue the whole count on `stream` and return.  d_out is DEVICE memory of at
 * least 16 uint64: [0..5] the counts, [6] the device self-check word (0 = fine; nonzero = a kernel's
 * consistency check fired and the counts are not valid, the case in which the blocking calls return
 * HARP_EDEVICE), [7] reserved, [8..15] the statistics.  It is written when the stream reaches that
 * point.  The handle's workspace is in use until then: do not start
 * another count on the same handle on a different stream before it completes. */
harp_status harp_count4_async(const harp_csr* g, const harp_plan* plan, uint64_t* d_out, void* stream);

/* Per-vertex (orbit) counts: for every vertex v and each of the HARP_NORBITS roles a vertex can play
 * in a connected induced 4-vertex motif, the number of induced occurrences S (Section II) that
 * contain v in that role.  The paper's closure (Section III-F) is global; this output refines it: a
 * role is the vertex's automorphism class in the motif (for 4-vertex motifs its degree inside
 * G[S] decides it), and the counts follow from eleven non-induced statistics per vertex (degree sums,
 * per-edge triangle counts, per-vertex triangles, 4-cycles and 4-cliques) by back-substitution in a
 * unit upper-triangular containment system, so they are exact modulo 2^64 like the global counts.
 * Summed over v, role r gives its motif's count times the number of the motif's vertices in r.
 *   orbits_out  uint64[n][HARP_NORBITS], row v = the input vertex id v; host memory if flags ==
 *               HARP_PTR_HOST, device memory if HARP_PTR_DEVICE.  Written only on HARP_OK.
 * Runs on the handle's stream and returns when the counts are in place.  The 4-cycle routing keeps
 * dense per-block counters of n uint32 (at most 4 GiB) for roots with more than 512 wedges.
 * Errors: HARP_EINVAL, HARP_ENOMEM, HARP_ECUDA, HARP_EDEVICE (a per-vertex sum failed its parity
 * check). */
enum {
    HARP_ORB_STAR_CENTER = 0, HARP_ORB_STAR_LEAF = 1, HARP_ORB_PATH_END = 2, HARP_ORB_PATH_INNER = 3,
    HARP_ORB_PAW_PENDANT = 4, HARP_ORB_PAW_HUB = 5, HARP_ORB_PAW_SIDE = 6, HARP_ORB_CYCLE = 7,
    HARP_ORB_DIAMOND_SPINE = 8, HARP_ORB_DIAMOND_TIP = 9, HARP_ORB_CLIQUE = 10, HARP_NORBITS = 11
};
harp_status harp_count4_orbits(const harp_csr* g, uint64_t* orbits_out, uint32_t flags);

/* Per-edge (edge orbit) counts: for every edge e and each of the HARP_NEDGE_ORBITS roles an edge can
 * play in a connected induced 4-vertex motif (decided by its endpoints' degrees inside G[S]), the
 * number of induced occurrences S whose G[S] contains e in that role.  Ten non-induced statistics per
 * edge (degree and triangle sums, triangles routed to their edges, 4-cycles routed from the wedge
 * walk to their edges, 4-cliques through the edge) and a unit upper-triangular containment system,
 * exact modulo 2^64.  Summed over the edges, role r gives its motif's count times the motif's edges
 * in r.
 *   orbits_out  uint64[m][HARP_NEDGE_ORBITS]; row k = the k-th edge (a, b), a < b, of the simple
 *               graph in lexicographic order of the input ids (the order of harp_csr_arrays' rows);
 *               host memory if flags == HARP_PTR_HOST, device memory if HARP_PTR_DEVICE.
 * Blocking on the handle's stream.  Errors as harp_count4_orbits. */
enum {
    HARP_EORB_STAR = 0, HARP_EORB_PATH_END = 1, HARP_EORB_PATH_MID = 2, HARP_EORB_PAW_PENDANT = 3,
    HARP_EORB_PAW_HUB = 4, HARP_EORB_PAW_FAR = 5, HARP_EORB_CYCLE = 6, HARP_EORB_DIAMOND_SPINE = 7,
    HARP_EORB_DIAMOND_RIM = 8, HARP_EORB_CLIQUE = 9, HARP_NEDGE_ORBITS = 10
};
harp_status harp_count4_edge_orbits(const harp_csr* g, uint64_t* orbits_out, uint32_t flags);

/* Connected induced 5-vertex motif counts (the paper's future work, Section VI): counts_out[21] (host)
 * in the order of the 21 connected 5-vertex classes.  Class order: a labelled graph on vertices 0..4
 * is a 10-bit mask, bit k for the k-th pair (i, j), i < j, in lexicographic order; its key is the
 * smallest mask over the 120 vertex permutations; the classes are numbered by increasing (edge count,
 * key) (harp_motif5_classes gives the keys).  Every connected 5-vertex subset is enumerated once on the
 * GPU (ESU rooted at each subset's lowest-ranked vertex) and classified by its adjacency mask; the work
 * is the number of connected 5-subsets, so this is for small and sparse graphs (a 5-vertex closure in
 * the manner of Section III-F is not built).  Scratch: 36 bytes x maximum degree per thread, at most
 * 4 GiB.  Blocking on the handle's stream.  Errors: HARP_EINVAL, HARP_ENOMEM, HARP_ECUDA. */
#define HARP_NMOTIFS5 21
harp_status harp_count5(const harp_csr* g, uint64_t counts_out[HARP_NMOTIFS5]);
/* The 21 class keys (10-bit canonical adjacency masks) in count order.  Host only (no device work). */
harp_status harp_motif5_classes(uint16_t keys_out[HARP_NMOTIFS5]);

/* Per-segment device times of the last count issued with profiling on (milliseconds, measured with
 * CUDA events recorded on the launching stream between the kernels).  Segments, in launch order:
 *   0 orientation (degree ranking, relabelled sorted CSR, out-CSR)
 *   1 triangle anchors, warp-local mode      2 triangle anchors, CTA mode (out-degree <= 256)
 *   3 triangle anchors, CTA mode (<= 1024)   4 triangle anchors, fallback (out-degree > 1024)
 *   5 wedge anchors, warp-local mode (+ work estimate of every root)
 *   6 wedge anchors, CTA hash mode           7 wedge anchors, windowed CTA mode
 *   8 reduction + closure
 * A count with the literal basis fills 0 (orientation), 1 (per-triangle X_j pass), 5 (per-edge
 * A_e x B_e pass) and 8 (per-vertex star pass + closure); the others read 0.
 * Call harp_set_profiling(1) first; the values are those of the last completed count.
 * launches_out receives the number of kernels the library launched in that count. */
#define HARP_NSEGMENTS 9
harp_status harp_set_profiling(int enable);
harp_status harp_last_stage_times(float ms_out[HARP_NSEGMENTS], int64_t* launches_out);

/* Total number of kernels the library has launched in this process. */
int64_t harp_launch_count(void);

/* ------------------------------------------------------------------------------------------------
 * Batched counting (thousands of graphs of uneven size).  The members' CSRs are packed into one
 * device arena (their disjoint union); every anchor's statistics go to its own member, so the whole
 * batch runs as one sequence of persistent kernels over global heavy-first work queues.  The
 * sequence is captured once into a CUDA graph and replayed by every harp_batch_count.
 * ---------------------------------------------------------------------------------------------- */
typedef struct harp_batch harp_batch;

/* Pack G handles (all on the current device) into a batch.  The members are copied; they may be
 * freed afterwards.  HARP_EOVERFLOW if the union exceeds 2^31-1 vertices or 2^32-1 arcs. */
harp_status harp_batch_create(const harp_csr* const* graphs, int64_t G, harp_batch** out);

/* Count every member; counts_out[G][6] (host) and optionally stats_out[G][8] (host, HARP_STAT_*
 * order).  The first call (and any call with a different plan) captures the CUDA graph; later calls
 * replay it on `stream` and return after the results are on the host.  plan->flags may carry
 * HARP_PLAN_NO_GRAPH to launch kernels one by one instead. */
harp_status harp_batch_count(harp_batch* b, const harp_plan* plan, uint64_t (*counts_out)[6],
                             uint64_t (*stats_out)[8], void* stream);

/* Number of members, union sizes and device bytes held by a batch.  Any output may be NULL. */
harp_status harp_batch_info(const harp_batch* b, int64_t* graphs, int64_t* n_total, int64_t* m_total,
                            size_t* device_bytes);

void harp_batch_free(harp_batch* b);

/* Autotuner for a batch: counts the batch `reps` times under each candidate plan (each captured as
 * its own CUDA graph, one untimed replay first), timed with CUDA events on the batch's stream, and
 * writes the fastest plan to *best and candidate k's mean milliseconds to ms_out[k] (may be NULL).
 * candidates NULL: the built-in per-degree-bin search, a coordinate descent from the default plan
 * that keeps the faster choice of each knob in turn: the warp/CTA split tri_warp_max {16, 32}; the
 * intersection variant of each triangle degree bin tri_probe_bin[k] {hash, bsearch}; the staging
 * capacity tri_cta_max {256, 512, 1024}; the wedge warp/CTA split c4_warp_max_work {256, 512}; the
 * wedge window c4_window_bytes {100, 200 KiB}.  At most HARP_AUTOTUNE_GRID plans are timed
 * (ms_out has that many entries, in the order timed, 0 past the last); identical plans are timed
 * once.  Otherwise ncand >= 1 given plans.  Every candidate must give identical counts and
 * statistics: a mismatch returns HARP_EDEVICE. */
#define HARP_AUTOTUNE_GRID 24
harp_status harp_batch_autotune(harp_batch* b, const harp_plan* candidates, int32_t ncand, int32_t reps,
                                harp_plan* best, float* ms_out);

/* One-shot convenience: create, count once (kernels launched directly), free. */
harp_status harp_count4_batch(const harp_csr* const* graphs, int64_t G, const harp_plan* plan,
                              uint64_t (*counts_out)[6], void* stream);

/* ------------------------------------------------------------------------------------------------
 * Ownership-preserving partitioned counting (Section III-E) for graphs whose counting footprint
 * exceeds a device-memory budget.  Rank space is cut into contiguous ranges; each range's halo (its
 * rows and those of its lower neighbours truncated below the range's end, and the out-lists of all
 * adjacent vertices) is copied to the device in turn, and only the anchors the range owns are
 * enumerated: an anchor's owner is the range of the first vertex of its globally ordered tuple (the
 * lowest vertex of a triangle / 4-clique anchor, the top vertex of a wedge anchor).  Per-edge
 * triangle counts are summed over ranges before sum_e C(t_e, 2); the closure runs once.
 * ---------------------------------------------------------------------------------------------- */
typedef struct harp_partition_stats {
    int64_t partitions;          /* ranges counted                                                */
    int64_t m;                   /* undirected simple edges                                       */
    int64_t halo_arcs;           /* arcs copied to the device over all ranges (rows + out-lists)  */
    uint64_t h2d_bytes;          /* host-to-device bytes over all ranges                          */
    uint64_t device_peak_bytes;  /* largest per-range device allocation                           */
    double host_ms;              /* host work: rank-order graph, range cuts, halo assembly, closure */
    double transfer_ms;          /* host <-> device copies (CUDA events around the copies)        */
    double device_ms;            /* counting kernels (CUDA events around the kernels)             */
    double graph_ms;             /* part of host_ms: the rank-order graph                         */
    double cut_ms;               /* part of host_ms: cutting the triangle ranges and wedge blocks */
    double tri_ms;               /* part of device_ms: triangle blocks                            */
    double wedge_ms;             /* part of device_ms: wedge blocks                               */
    int64_t tri_blocks;          /* triangle blocks (rank ranges)                                 */
    int64_t wedge_blocks;        /* wedge blocks ((rank range, x-slice) pairs)                    */
    int64_t wedge_sliced;        /* wedge blocks that hold only a slice of their range's x values */
} harp_partition_stats;

/* src, dst: HOST int32[m_in] (read only).  budget_bytes: device bytes one range may use (0 = half
 * of the free memory).  parts: > 0 forces that many equal rank ranges (tests); 0 sizes the ranges
 * to the budget, each the longest whose halo fits.  stats may be NULL.  Blocks until counts_out
 * (host) is filled.
 * Errors: HARP_EINVAL, HARP_EOVERFLOW, HARP_ENOMEM (the halo of some single vertex, or the
 * per-vertex arrays alone, exceed the budget; on hub-dominated graphs the 2-hop halo of the top
 * vertices approaches the whole graph), HARP_ECUDA, HARP_EDEVICE. */
harp_status harp_count4_partitioned(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                                    uint64_t budget_bytes, int32_t parts, uint64_t counts_out[6],
                                    harp_partition_stats* stats);

/* Host-only dry run of harp_count4_partitioned: builds the same rank-order graph and cuts the same
 * triangle ranges and wedge blocks under the same budget and parts rules, and counts nothing.  Lets a
 * caller see how many device passes a graph needs and the largest device allocation before it runs.
 * Ranges are in rank order (vertices sorted by (degree, id)), half-open.
 * stats (required) receives partitions, m, device_peak_bytes, tri_blocks, wedge_blocks, wedge_sliced,
 * graph_ms, cut_ms and host_ms (= graph_ms + cut_ms); the device and transfer fields are zero.
 * tri_out: HOST int64[2 * cap], the first cap triangle ranges as (lo, hi).  wedge_out: HOST
 * int64[4 * cap], the first cap wedge blocks as (root lo, root hi, x lo, x hi).  Both may be NULL when
 * cap = 0; compare stats->tri_blocks / wedge_blocks with cap to see whether all were written.
 * budget_bytes = 0 asks the device for half of its free memory, as the count does (HARP_ECUDA
 * without a device); with a budget > 0 no CUDA call is made.
 * Errors: HARP_EINVAL, HARP_EOVERFLOW, HARP_ENOMEM (as harp_count4_partitioned), HARP_ECUDA. */
harp_status harp_partition_plan(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                                uint64_t budget_bytes, int32_t parts, harp_partition_stats* stats,
                                int64_t* tri_out, int64_t* wedge_out, int64_t cap);

/* Host-only: the simple graph of a host edge list in global rank order, as the partitioned count
 * builds it on the host (Section III-D ordering): self-loops and duplicate edges dropped, vertices
 * sorted by (degree, id), every row of the symmetric CSR sorted ascending by rank.
 * m_out (required): undirected simple edges m.  rank_out: NULL or HOST int32[n], rank_out[v] = the
 * rank of input vertex v.  off_out: NULL or HOST int64[n+1], row offsets by rank.  cols_out: NULL or
 * HOST int32[cols_cap], the rows' ranks, written only when 2m <= cols_cap (call once with NULL to
 * learn m).  Errors: HARP_EINVAL (ids outside [0, n), negative sizes), HARP_EOVERFLOW, HARP_ENOMEM. */
harp_status harp_rank_csr_host(int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                               int64_t* m_out, int32_t* rank_out, int64_t* off_out, int32_t* cols_out,
                               int64_t cols_cap);

/* ------------------------------------------------------------------------------------------------
 * Serving with continuous batching.  Requests are admitted in arrival order while the device bytes
 * held by admitted requests stay within the HBM budget; their edge lists are copied and their CSRs
 * built on a copy stream while earlier batches count; every built request joins the next batch of
 * its lane (the batched pipeline, one launch per kernel).  Two lanes, each with its own executor
 * thread and compute stream: small requests (at most small_edges input pairs) on a higher-priority
 * stream, larger ones on the other, so a small request is not held behind a running large batch.  A request larger than the
 * budget is counted by the partitioned path under the budget.  Counts are exact and independent of
 * the mix a request was batched with.
 * ---------------------------------------------------------------------------------------------- */
typedef struct harp_server harp_server;

typedef struct harp_server_opts {
    uint64_t hbm_budget_bytes;   /* device bytes for admitted requests (0 = 64 GiB)              */
    uint32_t max_batch;          /* requests per batch (0 = 4096)                                */
    uint32_t max_inflight;       /* admitted but unfinished requests (0 = unlimited)            */
    uint32_t batch_window_us;    /* once a request is built, how long the executor may wait for  */
                                 /* requests still being admitted or built to join its batch    */
                                 /* (0 = launch at once with whatever is built)                 */
    uint32_t staging_mib;        /* page-locked host staging for submitted edge lists, MiB       */
                                 /* (0 = 512); a request that finds no room is kept in pageable */
                                 /* memory instead (slower host-to-device copy)                  */
    uint32_t small_edges;        /* requests of at most this many input pairs are batched and    */
                                 /* counted on a second, higher-priority compute stream, so they */
                                 /* do not wait behind a batch of large requests (0 = 65536;     */
                                 /* 0xFFFFFFFF = every request on one lane)                      */
} harp_server_opts;

typedef struct harp_server_stats {
    uint64_t completed, batches, batched_requests, partitioned, max_batch;
    uint64_t pending, resident_bytes, peak_resident_bytes;
    uint64_t latency_p50_us, latency_p99_us;  /* submit -> done, over the last 65,536 requests    */
} harp_server_stats;

/* Start a server on the current device (two builder threads with their own copy streams, one
 * executor thread with a compute stream).  opts may be NULL. */
harp_status harp_server_create(const harp_server_opts* opts, harp_server** out);

/* Enqueue a request; src/dst are HOST int32[m_in] and are copied before the call returns. */
harp_status harp_submit(harp_server* srv, int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                        uint64_t* ticket);

/* Non-blocking: *done = 0 while the request runs; *done = 1 once finished, in which case the
 * request's status is returned, counts_out is filled on HARP_OK and the ticket is retired (a ticket
 * belongs to one poller: the first poll or wait that sees it done retires it).
 * HARP_ENOTFOUND for an unknown or retired ticket. */
harp_status harp_poll(harp_server* srv, uint64_t ticket, uint64_t counts_out[6], int* done);

/* Blocking form of harp_poll; timeout_ms < 0 waits without limit, HARP_ETIMEOUT when it expires
 * (the request keeps running and can still be polled). */
harp_status harp_wait(harp_server* srv, uint64_t ticket, uint64_t counts_out[6], double timeout_ms);

harp_status harp_server_get_stats(harp_server* srv, harp_server_stats* out);

/* Stop the workers (after the batch on the GPU, if any) and free everything; unfinished requests
 * are dropped. */
void harp_server_destroy(harp_server* srv);

/* ------------------------------------------------------------------------------------------------
 * Counting without allocation.  The paper has no counterpart: this entry point exists for callers
 * that may not allocate device memory while they run (code inside another framework's
 * pre-reserved memory regime, services that forbid cudaMalloc/cudaFree after start-up because an
 * allocation can synchronise the device or fragment a sized pool, threads that only own a stream).
 *
 * harp_count4_noalloc counts the six induced motifs of a caller-owned, device-resident CSR:
 *   n, m       vertices and undirected simple edges; n <= 262,144 and m <= 524,288, larger sizes
 *              return HARP_ENOMEM (they do not fit the fixed scratch).  m must equal
 *              d_offsets[n] / 2.
 *   d_offsets  device int64[n+1], d_cols device int32[2m]: a symmetric CSR with every row sorted
 *              ascending, no self-loops, no duplicates (e.g. the arrays of harp_csr_arrays);
 *              read only.  The device checks d_offsets[0] = 0, d_offsets[n] = 2m, non-decreasing
 *              offsets with degrees <= n - 1 and column ids in [0, n) before anything else; a CSR
 *              that fails is counted as edgeless and d_out[6] is nonzero.  Self-loops, duplicates
 *              or an asymmetric CSR pass that check and give wrong counts.
 *   d_out      device uint64[16]: [0..5] counts, [6] the device self-check word (0 = fine; nonzero =
 *              the CSR check or a kernel's consistency check fired and the counts are not valid),
 *              [7] reserved, [8..15] statistics (HARP_STAT_* order), written when `stream` reaches
 *              the end of the work
 *   stream     cudaStream_t; the call only enqueues work and returns
 * Scratch lives in one file-scope static device array of 64 MiB that every GPU used by the process
 * holds until exit.  The first call on a device looks up that array's device address (once per
 * device, with the device current) and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this entry point again on a device after a
 * cudaDeviceReset of it.  All calls
 * share the array and clear what must start at zero themselves: calls whose work overlaps on the
 * GPU (different streams or threads) race on it, so serialise them.  No cudaMalloc, cudaFree or
 * allocating library routine is called. */
harp_status harp_count4_noalloc(int64_t n, int64_t m, const int64_t* d_offsets, const int32_t* d_cols,
                                uint64_t* d_out, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Errors.
 * ---------------------------------------------------------------------------------------------- */
const char* harp_status_str(harp_status s);
/* The last CUDA error code seen by this thread inside the library (0 if none) and its name. */
int harp_last_cuda_error(void);
const char* harp_last_cuda_error_str(void);

#ifdef __cplusplus
}
#endif
#endif /* HARP_H */
