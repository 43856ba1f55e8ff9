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

Parity status: pinned in ``tests/test_oracle_orbits.py`` (brute force over every 4-subset, closed forms
of complete, star, cycle, path, complete bipartite and wheel graphs, and the global counts of the C
oracle); nothing is pinned to a value printed in the paper, which prints no count.
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
