"""CPU oracle for connected induced 5-vertex motif counts.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may use it.  It shares no code with the CUDA library.

The paper counts 4-vertex motifs and names 5-vertex motifs as future work (Section VI).  An induced
occurrence of a k-vertex motif is a k-vertex subset S with G[S] connected (Section II); here k = 5.
The classes are the isomorphism classes of connected graphs on five vertices.  Each labelled graph
on vertices 0..4 is a 10-bit mask over the pairs (i, j), i < j, in lexicographic order; its class key
is the smallest mask over the 120 vertex permutations.  :data:`CLASSES` lists the keys of the
connected classes in increasing order (edge count first); counts follow that order.

Functions: :func:`count5_brute` (every 5-subset) and :func:`count5_esu` (each connected 5-set once,
Wernicke's ESU).

Parity status: pinned in ``tests/test_oracle_motifs5.py`` (the class table against the known numbers
of connected graphs on five vertices, 21 unlabelled and 728 labelled, and orbit-stabiliser sizes;
closed forms of complete, star, cycle, path and complete bipartite graphs; each class's own graph
alone; ESU against brute force; class totals against the number of connected 5-subsets); nothing is
pinned to a value printed in the paper, which prints no count.
"""
from __future__ import annotations

import itertools

import numpy as np

PAIRS = tuple(itertools.combinations(range(5), 2))
_BIT = {p: k for k, p in enumerate(PAIRS)}


def _mask(edges):
    m = 0
    for a, b in edges:
        m |= 1 << _BIT[(min(a, b), max(a, b))]
    return m


def _edges_of(mask):
    return [p for k, p in enumerate(PAIRS) if mask >> k & 1]


def _connected(mask):
    adj = {v: set() for v in range(5)}
    for a, b in _edges_of(mask):
        adj[a].add(b)
        adj[b].add(a)
    seen, stack = {0}, [0]
    while stack:
        for y in adj[stack.pop()]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen) == 5


def _canonical(mask):
    edges = _edges_of(mask)
    return min(_mask([(p[a], p[b]) for a, b in edges]) for p in itertools.permutations(range(5)))


# class key of every labelled 5-vertex graph (None when disconnected)
_CANON = [(_canonical(m) if _connected(m) else None) for m in range(1 << len(PAIRS))]
CLASSES = tuple(sorted({c for c in _CANON if c is not None}, key=lambda c: (bin(c).count("1"), c)))
_INDEX = {c: i for i, c in enumerate(CLASSES)}


def class_edges(i):
    """Edges of a representative graph of class i (vertices 0..4)."""
    return _edges_of(CLASSES[i])


def _class_of(adj, s):
    m = 0
    for k, (a, b) in enumerate(PAIRS):
        if s[b] in adj[s[a]]:
            m |= 1 << k
    c = _CANON[m]
    return None if c is None else _INDEX[c]


def _adjacency(n, src, dst):
    adj = [set() for _ in range(n)]
    for a, b in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if not (0 <= a < n and 0 <= b < n):
            raise ValueError("vertex id outside [0, n)")
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def count5_brute(n, src, dst):
    """The definition over every 5-subset of [0, n) (tiny graphs only)."""
    adj = _adjacency(n, src, dst)
    out = np.zeros(len(CLASSES), np.uint64)
    for s in itertools.combinations(range(n), 5):
        c = _class_of(adj, s)
        if c is not None:
            out[c] += 1
    return out


def count5_esu(n, src, dst):
    """The same counts, with each connected 5-set enumerated once by Wernicke's ESU (2006): a root v is
    extended only by vertices above v that are exclusive neighbours of the newest vertex."""
    adj = _adjacency(n, src, dst)
    out = np.zeros(len(CLASSES), np.uint64)

    def extend(sub, ext, root):
        if len(sub) == 5:
            out[_class_of(adj, sub)] += 1
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


def class_of_edges(edges):
    """Class index of the connected graph on vertices 0..4 with the given edges."""
    c = _CANON[_mask(edges)]
    if c is None:
        raise ValueError("not a connected graph on five vertices")
    return _INDEX[c]
