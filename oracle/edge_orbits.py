"""CPU oracle for per-edge (edge orbit) counts of connected induced 4-vertex motifs.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may use it.  It shares no code with the CUDA library.

The per-edge refinement of an induced occurrence S (Section II) assigns each edge of G[S] the class of
edges an automorphism of the motif maps it to.  For the six 4-vertex motifs the class is decided by
the degrees of its two endpoints inside G[S]:

    edge orbit          motif     endpoint degrees in G[S]   edges of the motif in it
    star_edge           3-star    3, 1                       3
    path_end_edge       4-path    2, 1                       2
    path_mid_edge       4-path    2, 2                       1
    paw_pendant_edge    paw       3, 1                       1
    paw_hub_edge        paw       3, 2                       2
    paw_far_edge        paw       2, 2                       1
    cycle_edge          4-cycle   2, 2                       4
    diamond_spine_edge  diamond   3, 3                       1
    diamond_rim_edge    diamond   3, 2                       4
    clique_edge         4-clique  3, 3                       6

``out[k, o]`` = number of induced occurrences S whose subgraph G[S] contains edge k and in which that
edge is in orbit o; edges are numbered as :func:`edge_list` returns them.  Summed over edges, orbit o
gives its motif's count times its number of edges (the last column).

Functions: :func:`edge_orbits4_brute` (every 4-subset), :func:`edge_orbits4_esu` (each connected 4-set
once) and :func:`edge_orbits4_combo` (ten non-induced statistics per edge and a unit upper-triangular
containment inversion).

Parity status: pinned in ``tests/test_oracle_edge_orbits.py`` (each motif graph alone, closed forms of
complete, star, cycle, path and complete bipartite graphs, ESU against brute force, edge-orbit sums
against the C oracle's global counts, and the vertex orbits of ``oracle.orbits``); nothing is pinned
to a value printed in the paper, which prints no count.
"""
from __future__ import annotations

import itertools

import numpy as np

EDGE_ORBITS = ("star_edge", "path_end_edge", "path_mid_edge", "paw_pendant_edge", "paw_hub_edge",
               "paw_far_edge", "cycle_edge", "diamond_spine_edge", "diamond_rim_edge", "clique_edge")
# motif index (order star3, path4, paw, cycle4, diamond, clique4) and edges of the motif in each orbit
EDGE_ORBIT_MOTIF = (0, 1, 1, 2, 2, 2, 3, 4, 4, 5)
EDGE_ORBIT_SIZE = (3, 2, 1, 1, 2, 1, 4, 1, 4, 6)


def edge_list(n, src, dst):
    """The simple graph's edges (a, b), a < b, in increasing order; ids outside [0, n) raise."""
    pairs = set()
    for a, b in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if not (0 <= a < n and 0 <= b < n):
            raise ValueError("vertex id outside [0, n)")
        if a != b:
            pairs.add((min(a, b), max(a, b)))
    return sorted(pairs)


def _edge_roles(adj, s):
    """[(edge, orbit)] for the edges of G[s], or None when G[s] is not connected."""
    deg = {x: sum(1 for y in s if y in adj[x]) for x in s}
    edges = [(a, b) for a, b in itertools.combinations(sorted(s), 2) if b in adj[a]]
    if len(edges) < 3:
        return None
    dmax = max(deg.values())
    if len(edges) == 3:
        if dmax == 3:
            motif = "star"
        elif sorted(deg.values()) == [1, 1, 2, 2]:
            motif = "path"
        else:
            return None  # a triangle and an isolated vertex
    elif len(edges) == 4:
        motif = "paw" if dmax == 3 else "cycle"
    elif len(edges) == 5:
        motif = "diamond"
    else:
        motif = "clique"
    out = []
    for a, b in edges:
        hi, lo = max(deg[a], deg[b]), min(deg[a], deg[b])
        if motif == "star":
            o = 0
        elif motif == "path":
            o = 1 if lo == 1 else 2
        elif motif == "paw":
            o = 3 if lo == 1 else (4 if hi == 3 else 5)
        elif motif == "cycle":
            o = 6
        elif motif == "diamond":
            o = 7 if lo == 3 else 8
        else:
            o = 9
        out.append(((a, b), o))
    return out


def _adjacency(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    return adj


def edge_orbits4_brute(n, src, dst):
    """The definition over every 4-subset of [0, n) (tiny graphs only)."""
    edges = edge_list(n, src, dst)
    index = {e: k for k, e in enumerate(edges)}
    adj = _adjacency(n, edges)
    out = np.zeros((len(edges), len(EDGE_ORBITS)), np.uint64)
    for s in itertools.combinations(range(n), 4):
        r = _edge_roles(adj, s)
        if r is not None:
            for e, o in r:
                out[index[e], o] += 1
    return out


def edge_orbits4_esu(n, src, dst):
    """The same counts, with each connected 4-set enumerated once by Wernicke's ESU (2006)."""
    edges = edge_list(n, src, dst)
    index = {e: k for k, e in enumerate(edges)}
    adj = _adjacency(n, edges)
    out = np.zeros((len(edges), len(EDGE_ORBITS)), np.uint64)

    def extend(sub, ext, root):
        if len(sub) == 4:
            for e, o in _edge_roles(adj, sub):
                out[index[e], o] += 1
            return
        ext = list(ext)
        closed = set(sub)
        for x in sub:
            closed |= adj[x]
        while ext:
            w = ext.pop()
            excl = [y for y in adj[w] if y > root and y not in closed]
            extend(sub + [w], ext + excl, root)

    for v in range(n):
        extend([v], [y for y in adj[v] if y > v], v)
    return out


# ---------------------------------------------------------------------------------------------------
# Per-edge closure: ten non-induced statistics per edge e = (a, b) and their containment system.
# ---------------------------------------------------------------------------------------------------
# E[i] counts (not necessarily induced) copies of a pattern that contain e in role i; an induced
# occurrence S containing e contributes the number of such copies inside G[S].  Row i gives that
# number for each edge orbit (columns in EDGE_ORBITS order); the matrix is unit upper triangular.
#   E0  stars containing e                           C(d_a - 1, 2) + C(d_b - 1, 2)
#   E1  3-edge paths with e at an end                sum over the two orientations (a end, b inner) of
#                                                    sum_{c in N(b), c != a} (d_c - 1) - t_ab
#   E2  3-edge paths with e in the middle            (d_a - 1)(d_b - 1) - t_ab
#   E3  paws with e the pendant edge                 (t_a - t_ab) + (t_b - t_ab)
#   E4  paws with e a triangle edge at the hub       t_ab (d_a + d_b - 4)
#   E5  paws with e the triangle edge facing the hub sum_{h in N(a) n N(b)} (d_h - 2)
#   E6  4-cycles through e                           sum_{x in N(a), x != b} (|N(x) n N(b)| - 1)
#   E7  diamonds with e the shared edge              C(t_ab, 2)
#   E8  diamonds with e an outer edge                sum_{s in N(a) n N(b)} (t_as - 1) + (t_bs - 1)
#   E9  4-cliques through e                          edges of G[N(a) n N(b)]
# with t_e = triangles on edge e and t_v = triangles on vertex v.
EDGE_CONTAINMENT = np.array([
    # o0 o1 o2 o3 o4 o5 o6 o7 o8 o9
    [1, 0, 0, 1, 1, 0, 0, 2, 1, 2],   # E0: endpoints of e of degree 3 in G[S]
    [0, 1, 0, 2, 0, 2, 2, 0, 3, 4],   # E1: Hamiltonian paths of G[S] ending with e
    [0, 0, 1, 0, 1, 0, 1, 2, 1, 2],   # E2: Hamiltonian paths of G[S] with e in the middle
    [0, 0, 0, 1, 0, 0, 0, 0, 1, 2],   # E3
    [0, 0, 0, 0, 1, 0, 0, 4, 1, 4],   # E4
    [0, 0, 0, 0, 0, 1, 0, 0, 1, 2],   # E5
    [0, 0, 0, 0, 0, 0, 1, 0, 1, 2],   # E6
    [0, 0, 0, 0, 0, 0, 0, 1, 0, 1],   # E7
    [0, 0, 0, 0, 0, 0, 0, 0, 1, 4],   # E8
    [0, 0, 0, 0, 0, 0, 0, 0, 0, 1],   # E9
], dtype=np.int64)


def noninduced_per_edge(n, src, dst):
    """The ten statistics E0..E9 of every edge (in edge_list order), by plain loops."""
    edges = edge_list(n, src, dst)
    adj = _adjacency(n, edges)
    deg = [len(x) for x in adj]
    t = {e: len(adj[e[0]] & adj[e[1]]) for e in edges}

    def te(x, y):
        return t[(x, y) if x < y else (y, x)]

    t_v = [sum(te(v, h) for h in adj[v]) // 2 for v in range(n)]
    out = np.zeros((len(edges), 10), np.uint64)
    for k, (a, b) in enumerate(edges):
        common = adj[a] & adj[b]
        tab = len(common)
        E = [0] * 10
        E[0] = (deg[a] - 1) * (deg[a] - 2) // 2 + (deg[b] - 1) * (deg[b] - 2) // 2
        E[1] = sum(sum(deg[c] - 1 for c in adj[y] if c != x) - tab for x, y in ((a, b), (b, a)))
        E[2] = (deg[a] - 1) * (deg[b] - 1) - tab
        E[3] = (t_v[a] - tab) + (t_v[b] - tab)
        E[4] = tab * (deg[a] + deg[b] - 4)
        E[5] = sum(deg[h] - 2 for h in common)
        E[6] = sum(len(adj[x] & adj[b]) - 1 for x in adj[a] if x != b)
        E[7] = tab * (tab - 1) // 2
        E[8] = sum((te(a, s) - 1) + (te(b, s) - 1) for s in common)
        E[9] = sum(1 for x in common for y in common if x < y and y in adj[x])
        out[k] = E
    return out


def edge_orbits4_combo(n, src, dst):
    """Edge-orbit counts by back-substitution in the per-edge containment system (mod 2^64)."""
    N = noninduced_per_edge(n, src, dst)
    out = np.zeros(N.shape, np.uint64)
    for k in range(N.shape[0]):
        o = [0] * 10
        for i in range(9, -1, -1):
            o[i] = int(N[k, i]) - sum(int(EDGE_CONTAINMENT[i, j]) * o[j] for j in range(i + 1, 10))
        out[k] = [x % (1 << 64) for x in o]
    return out
