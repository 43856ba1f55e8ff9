"""The host work meter (the numerators of the bench's roofline figures) against brute force.

The meter counts work with vectorised numpy; here the same quantities are counted by plain loops over
the rank-ordered graph on small inputs: ordered wedges of the 4-cycle anchor (root u, lower neighbour
w, opposite vertex x of degree >= 2 below u) and probed elements of the triangle anchor (for every
out-arc (u, v) except the last of N+(u): the elements of N+(v) up to max N+(u)).
"""
import numpy as np
import pytest

import graphgen
from paper_2607_12074_gb300 import workmeter


def rank_adjacency(n, src, dst):
    pairs = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist()) if a != b}
    deg = [0] * n
    for a, b in pairs:
        deg[a] += 1
        deg[b] += 1
    order = sorted(range(n), key=lambda v: (deg[v], v))
    rank = {v: r for r, v in enumerate(order)}
    adj = [set() for _ in range(n)]
    for a, b in pairs:
        adj[rank[a]].add(rank[b])
        adj[rank[b]].add(rank[a])
    return [sorted(s) for s in adj]


def brute_wedges(adj):
    n = len(adj)
    n1 = next((r for r in range(n) if len(adj[r]) >= 2), n)
    total = 0
    per_root = [0] * n
    for u in range(n):
        for w in adj[u]:
            if w < u:
                c = sum(1 for x in adj[w] if n1 <= x < u)
                per_root[u] += c
                total += c
    return total, per_root


def brute_probes(adj):
    total = 0
    for u, row in enumerate(adj):
        out = [v for v in row if v > u]
        if not out:
            continue
        top = out[-1]
        for v in out[:-1]:
            total += sum(1 for y in adj[v] if y > v and y <= top)
    return total


GRAPHS = {
    "ba": lambda: graphgen.ba(400, 5, 3),
    "er": lambda: graphgen.er(300, 6.0, 4),
    "rmat": lambda: graphgen.rmat(9, 8, seed=2),
    "rgg": lambda: graphgen.rgg(400, 8.0, 5),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_wedge_and_probe_totals(name):
    g = GRAPHS[name]()
    adj = rank_adjacency(g.n, g.src, g.dst)
    m = workmeter.meter(g.n, g.src, g.dst)
    total, per_root = brute_wedges(adj)
    assert m["c4_wedges_total"] == total
    assert m["tri_probes_total"] == brute_probes(adj)
    # roots with fewer than two lower neighbours close no 4-cycle and take no tier
    dm = [sum(1 for x in adj[u] if x < u) for u in range(len(adj))]
    tiers = ("c4_small", "c4_mid", "c4_window")
    assert sum(m[t]["wedges"] for t in tiers) == sum(w for u, w in enumerate(per_root) if dm[u] >= 2)
    assert sum(m[t]["roots"] for t in tiers) == sum(1 for u, w in enumerate(per_root) if w > 0 and dm[u] >= 2)
    assert m["c4_small"]["items"] == m["c4_small"]["roots"]
    assert m["c4_window"]["items"] >= m["c4_window"]["roots"]
    assert m["m"] == sum(len(r) for r in adj) // 2


def test_warp_limit_moves_roots_to_the_windows():
    """Roots with work W(u) <= the warp limit take the warp hash, those up to the middle limit the
    middle tier's larger hash, the rest the windowed counters."""
    g = graphgen.ba(400, 5, 3)
    adj = rank_adjacency(g.n, g.src, g.dst)
    _, per_root = brute_wedges(adj)
    dm = [sum(1 for x in adj[u] if x < u) for u in range(len(adj))]
    for limit, mid in ((1, 1), (16, 16), (64, 64), (16, 200), (64, 2048)):
        m = workmeter.meter(g.n, g.src, g.dst, c4_warp_max=limit, c4_mid_max=mid)
        assert m["c4_window"]["wedges"] == sum(w for u, w in enumerate(per_root) if dm[u] >= 2 and w > mid)
        assert m["c4_mid"]["wedges"] == sum(w for u, w in enumerate(per_root) if dm[u] >= 2 and limit < w <= mid)
        assert m["c4_mid"]["items"] == m["c4_mid"]["roots"]
        assert m["c4_small"]["wedges"] == sum(w for u, w in enumerate(per_root) if dm[u] >= 2 and 0 < w <= limit)
