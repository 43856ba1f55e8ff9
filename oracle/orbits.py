"""CPU oracle for per-vertex (orbit) counts of connected induced 4-vertex motifs.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may use it.  It shares no code with the CUDA library.

The paper derives global counts only (Section III-F); a per-vertex output refines each induced
occurrence S (Section II: a 4-vertex subset whose induced subgraph is connected) by the role each of
its vertices plays.  Two vertices play the same role when an automorphism of the motif maps one to the
other, which for the six 4-vertex motifs is decided by the vertex's degree inside G[S]:

    orbit              motif     degree in G[S]   vertices of the motif in it
    star_center        3-star    3                1
    star_leaf          3-star    1                3
    path_end           4-path    1                2
    path_inner         4-path    2                2
    paw_pendant        paw       1                1
    paw_hub            paw       3                1
    paw_side           paw       2                2
    cycle              4-cycle   2                4
    diamond_spine      diamond   3                2
    diamond_tip        diamond   2                2
    clique             4-clique  3                4

``out[v, o]`` = number of induced occurrences S with v in S playing orbit o.  Summed over v, orbit o
gives its motif's count times the number of its vertices in that orbit (the last column).

Functions: :func:`orbits4_brute` (every 4-subset), :func:`orbits4_esu` (each connected 4-set once) and
:func:`orbits4_combo` (eleven non-induced statistics per vertex and a unit upper-triangular
containment inversion, the per-vertex analogue of the global closure of Section III-F).

Parity status: pinned in ``tests/test_oracle_orbits.py`` (brute force over every 4-subset, closed forms
of complete, star, cycle, path, complete bipartite and wheel graphs, each motif graph alone, and the
global counts of the C oracle); nothing is pinned to a value printed in the paper, which prints no
count.
"""
from __future__ import annotations

import itertools

import numpy as np

ORBITS = ("star_center", "star_leaf", "path_end", "path_inner", "paw_pendant", "paw_hub", "paw_side", "cycle",
          "diamond_spine", "diamond_tip", "clique")
# motif index (order star3, path4, paw, cycle4, diamond, clique4) and vertices of the motif in each orbit
ORBIT_MOTIF = (0, 0, 1, 1, 2, 2, 2, 3, 4, 4, 5)
ORBIT_SIZE = (1, 3, 2, 2, 1, 1, 2, 4, 2, 2, 4)


def _adjacency(n, src, dst):
    adj = [set() for _ in range(n)]
    for a, b in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if not (0 <= a < n and 0 <= b < n):
            raise ValueError("vertex id outside [0, n)")
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def _roles(adj, s):
    """Orbit of each vertex of the 4-set s, or None when G[s] is not connected."""
    deg = [sum(1 for y in s if y in adj[x]) for x in s]
    edges = sum(deg) // 2
    if edges < 3:
        return None  # three edges at least are needed to connect four vertices
    if edges == 3:
        if max(deg) == 3:
            return [0 if d == 3 else 1 for d in deg]  # star: centre and leaves
        if deg.count(1) == 2:
            return [2 if d == 1 else 3 for d in deg]  # path: ends and inner vertices
        return None  # a triangle and an isolated vertex
    if edges == 4:
        if max(deg) == 3:
            return [4 if d == 1 else (5 if d == 3 else 6) for d in deg]  # paw
        return [7] * 4  # every degree 2: the 4-cycle
    if edges == 5:
        return [8 if d == 3 else 9 for d in deg]  # diamond
    return [10] * 4


def orbits4_brute(n, src, dst):
    """The definition over every 4-subset of [0, n) (tiny graphs only)."""
    adj = _adjacency(n, src, dst)
    out = np.zeros((n, len(ORBITS)), np.uint64)
    for s in itertools.combinations(range(n), 4):
        r = _roles(adj, s)
        if r is not None:
            for v, o in zip(s, r):
                out[v, o] += 1
    return out


def orbits4_esu(n, src, dst):
    """The same counts, with each connected 4-set enumerated once by Wernicke's ESU (2006): a root v
    is extended only by vertices above v that are exclusive neighbours of the newest vertex."""
    adj = _adjacency(n, src, dst)
    out = np.zeros((n, len(ORBITS)), np.uint64)

    def extend(sub, ext, root):
        if len(sub) == 4:
            for v, o in zip(sub, _roles(adj, sub)):
                out[v, o] += 1
            return
        ext = list(ext)
        closed = set(sub)
        for x in sub:
            closed |= adj[x]
        while ext:
            w = ext.pop()
            # exclusive neighbours of w: above the root, not in the subgraph or its neighbourhood
            excl = [y for y in adj[w] if y > root and y not in closed]
            extend(sub + [w], ext + excl, root)

    for v in range(n):
        extend([v], [y for y in adj[v] if y > v], v)
    return out


# ---------------------------------------------------------------------------------------------------
# Per-vertex closure: eleven non-induced statistics per vertex and their containment system.
# ---------------------------------------------------------------------------------------------------
# N[i] counts (not necessarily induced) copies of a pattern in which v plays role i; every induced
# occurrence S that contains v contributes the number of such copies inside G[S].  Row i lists the
# contribution of each induced orbit o (columns in ORBITS order); the matrix is unit upper triangular,
# so the orbits follow by back-substitution from the 4-clique up, without division.
#   N0  stars centred at v                         C(d_v, 3)
#   N1  stars with v a leaf                        sum_{c in N(v)} C(d_c - 1, 2)
#   N2  3-edge paths with v an end                 sum_{a in N(v)} sum_{b in N(a), b != v} (d_b - 1 - [b ~ v])
#   N3  3-edge paths with v inner                  sum_{b in N(v)} sum_{a in N(v), a != b} (d_b - 1 - [a ~ b])
#   N4  paws with v the pendant                    sum_{h in N(v)} (t_h - t_vh)
#   N5  paws with v the degree-3 vertex            t_v (d_v - 2)
#   N6  paws with v a degree-2 triangle vertex     sum_{h in N(v)} t_vh (d_h - 2)
#   N7  4-cycles through v                         sum_{x != v} C(|N(v) n N(x)|, 2)
#   N8  diamonds with v on the shared edge         sum_{s in N(v)} C(t_vs, 2)
#   N9  diamonds with v a degree-2 vertex          sum_{triangles {v, a, b}} (t_ab - 1)
#   N10 4-cliques through v
# with t_e = triangles on edge e and t_v = triangles on vertex v.
CONTAINMENT = np.array([
    # o0 o1 o2 o3 o4 o5 o6 o7 o8 o9 o10
    [1, 0, 0, 0, 0, 1, 0, 0, 1, 0, 1],   # N0: v of degree 3 in G[S]
    [0, 1, 0, 0, 1, 0, 1, 0, 1, 2, 3],   # N1: neighbours of v of degree 3 in G[S]
    [0, 0, 1, 0, 2, 0, 1, 2, 2, 4, 6],   # N2: Hamiltonian paths of G[S] ending at v
    [0, 0, 0, 1, 0, 2, 1, 2, 4, 2, 6],   # N3: Hamiltonian paths of G[S] through v
    [0, 0, 0, 0, 1, 0, 0, 0, 0, 2, 3],   # N4
    [0, 0, 0, 0, 0, 1, 0, 0, 2, 0, 3],   # N5
    [0, 0, 0, 0, 0, 0, 1, 0, 2, 2, 6],   # N6
    [0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 3],   # N7
    [0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 3],   # N8
    [0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 3],   # N9
    [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1],   # N10
], dtype=np.int64)


def noninduced_per_vertex(n, src, dst):
    """The eleven statistics N0..N10 of every vertex, by plain loops over the simple graph."""
    adj = _adjacency(n, src, dst)
    deg = [len(a) for a in adj]
    t_e = {}
    for u in range(n):
        for v in adj[u]:
            if u < v:
                t_e[(u, v)] = len(adj[u] & adj[v])

    def te(a, b):
        return t_e[(a, b) if a < b else (b, a)]

    t_v = [sum(te(v, h) for h in adj[v]) // 2 for v in range(n)]
    out = np.zeros((n, 11), np.uint64)
    for v in range(n):
        d = deg[v]
        N = [0] * 11
        N[0] = d * (d - 1) * (d - 2) // 6
        N[1] = sum((deg[c] - 1) * (deg[c] - 2) // 2 for c in adj[v])
        N[2] = sum(deg[b] - 1 - (b in adj[v]) for a in adj[v] for b in adj[a] if b != v)
        N[3] = sum(deg[b] - 1 - (a in adj[b]) for b in adj[v] for a in adj[v] if a != b)
        N[4] = sum(t_v[h] - te(v, h) for h in adj[v])
        N[5] = t_v[v] * (d - 2) if d >= 2 else 0
        N[6] = sum(te(v, h) * (deg[h] - 2) for h in adj[v])
        common = {}
        for a in adj[v]:
            for x in adj[a]:
                if x != v:
                    common[x] = common.get(x, 0) + 1
        N[7] = sum(c * (c - 1) // 2 for c in common.values())
        N[8] = sum(te(v, s) * (te(v, s) - 1) // 2 for s in adj[v])
        N[9] = sum(te(a, b) - 1 for a in adj[v] for b in adj[v] if a < b and b in adj[a])
        N[10] = sum(1 for a in adj[v] for b in adj[v] for c in adj[v]
                    if a < b < c and b in adj[a] and c in adj[a] and c in adj[b])
        out[v] = N
    return out


def orbits4_combo(n, src, dst):
    """Orbit counts by back-substitution in the per-vertex containment system (mod 2^64)."""
    N = noninduced_per_vertex(n, src, dst).astype(object)
    out = np.zeros((n, 11), np.uint64)
    for v in range(n):
        o = [0] * 11
        for i in range(10, -1, -1):
            o[i] = int(N[v, i]) - sum(int(CONTAINMENT[i, j]) * o[j] for j in range(i + 1, 11))
        out[v] = [x % (1 << 64) for x in o]
    return out
