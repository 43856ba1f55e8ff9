"""Pins of the per-edge (edge orbit) oracle: each motif graph alone, closed forms, ESU against brute force,
the C oracle's global counts and the per-vertex orbits."""
import math
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle as O
from oracle import edge_orbits as E
from oracle import orbits as V

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import complete, cycle, kbip, path, star  # noqa: E402

C = math.comb
IDX = {name: i for i, name in enumerate(E.EDGE_ORBITS)}


def per_edge(n, s, d, want):
    """Array [m, 10] from {(a, b): {orbit name: count}} over the graph's edge list."""
    edges = E.edge_list(n, s, d)
    out = np.zeros((len(edges), len(E.EDGE_ORBITS)), np.uint64)
    for k, e in enumerate(edges):
        for name, c in want(e).items():
            out[k, IDX[name]] = c
    return out


def both(n, s, d):
    a, b = E.edge_orbits4_brute(n, s, d), E.edge_orbits4_esu(n, s, d)
    assert np.array_equal(a, b)
    return a


def test_orbit_table_is_consistent():
    edges_per_motif = (3, 3, 4, 4, 5, 6)
    for motif in range(6):
        assert sum(k for o, k in zip(E.EDGE_ORBIT_MOTIF, E.EDGE_ORBIT_SIZE) if o == motif) == edges_per_motif[motif]


# each motif graph alone: every edge's class read off the drawing
MOTIF_GRAPHS = {
    "star": {(0, 1): "star_edge", (0, 2): "star_edge", (0, 3): "star_edge"},
    "path": {(0, 1): "path_end_edge", (1, 2): "path_mid_edge", (2, 3): "path_end_edge"},
    "paw": {(0, 1): "paw_hub_edge", (0, 2): "paw_hub_edge", (1, 2): "paw_far_edge", (0, 3): "paw_pendant_edge"},
    "cycle": {(0, 1): "cycle_edge", (1, 2): "cycle_edge", (2, 3): "cycle_edge", (0, 3): "cycle_edge"},
    "diamond": {(0, 1): "diamond_spine_edge", (0, 2): "diamond_rim_edge", (0, 3): "diamond_rim_edge",
                (1, 2): "diamond_rim_edge", (1, 3): "diamond_rim_edge"},
    "clique": {(a, b): "clique_edge" for a in range(4) for b in range(a + 1, 4)},
}


@pytest.mark.parametrize("name", sorted(MOTIF_GRAPHS))
def test_each_motif_graph_alone(name):
    roles = MOTIF_GRAPHS[name]
    perm = [3, 1, 0, 2]  # so the classes do not follow vertex order
    relabel = {tuple(sorted((perm[a], perm[b]))): r for (a, b), r in roles.items()}
    s = np.array([a for a, _ in relabel], np.int32)
    d = np.array([b for _, b in relabel], np.int32)
    assert np.array_equal(both(4, s, d), per_edge(4, s, d, lambda e: {relabel[e]: 1}))


@pytest.mark.parametrize("n", [4, 5, 7])
def test_complete_graph(n):
    s, d = complete(n)
    assert np.array_equal(both(n, s, d), per_edge(n, s, d, lambda e: {"clique_edge": C(n - 2, 2)}))


@pytest.mark.parametrize("k", [3, 5])
def test_star(k):
    s, d = star(k)
    assert np.array_equal(both(k + 1, s, d), per_edge(k + 1, s, d, lambda e: {"star_edge": C(k - 1, 2)}))


@pytest.mark.parametrize("n", [4, 5, 8])
def test_cycle(n):
    s, d = cycle(n)
    want = (lambda e: {"cycle_edge": 1}) if n == 4 else (lambda e: {"path_end_edge": 2, "path_mid_edge": 1})
    assert np.array_equal(both(n, s, d), per_edge(n, s, d, want))


@pytest.mark.parametrize("n", [4, 6, 9])
def test_path(n):
    s, d = path(n)

    def want(e):
        i = e[0]  # edge (i, i + 1): middle of the window i-1..i+2, an end of i..i+3 and of i-2..i+1
        return {"path_mid_edge": int(i >= 1 and i + 2 <= n - 1), "path_end_edge": int(i + 3 <= n - 1) + int(i >= 2)}
    assert np.array_equal(both(n, s, d), per_edge(n, s, d, want))


@pytest.mark.parametrize("a,b", [(2, 3), (3, 4), (4, 4)])
def test_complete_bipartite(a, b):
    s, d = kbip(a, b)
    # an edge is in the stars centred at either endpoint and the 4-cycles through one more vertex per side
    want = {"star_edge": C(a - 1, 2) + C(b - 1, 2), "cycle_edge": (a - 1) * (b - 1)}
    assert np.array_equal(both(a + b, s, d), per_edge(a + b, s, d, lambda e: want))


@pytest.mark.parametrize("seed", range(10))
def test_esu_equals_brute_force_on_random_graphs(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(5, 13))
    p = float(rng.uniform(0.15, 0.8))
    pairs = [(x, y) for x in range(n) for y in range(x + 1, n) if rng.random() < p]
    s = np.array([x for x, _ in pairs], np.int32)
    d = np.array([y for _, y in pairs], np.int32)
    both(n, s, d)


# edges of each edge orbit incident to a vertex of each vertex orbit (one occurrence)
INCIDENT = np.zeros((len(V.ORBITS), len(E.EDGE_ORBITS)), np.int64)
for vo, eo, k in [("star_center", "star_edge", 3), ("star_leaf", "star_edge", 1),
                  ("path_end", "path_end_edge", 1), ("path_inner", "path_end_edge", 1), ("path_inner", "path_mid_edge", 1),
                  ("paw_pendant", "paw_pendant_edge", 1), ("paw_hub", "paw_pendant_edge", 1), ("paw_hub", "paw_hub_edge", 2),
                  ("paw_side", "paw_hub_edge", 1), ("paw_side", "paw_far_edge", 1), ("cycle", "cycle_edge", 2),
                  ("diamond_spine", "diamond_spine_edge", 1), ("diamond_spine", "diamond_rim_edge", 2),
                  ("diamond_tip", "diamond_rim_edge", 2), ("clique", "clique_edge", 3)]:
    INCIDENT[V.ORBITS.index(vo), IDX[eo]] = k


@pytest.mark.parametrize("name,make", [("ba", lambda: graphgen.ba(120, 3, 2)), ("rgg", lambda: graphgen.rgg(120, 6.0, 4)),
                                       ("rmat", lambda: graphgen.rmat(7, 8, seed=3))])
def test_edge_orbits_against_vertex_orbits_and_global_counts(name, make):
    """Per vertex, the edge orbits of its incident edges add up to its vertex orbits times the incidence
    table; summed over edges, each edge orbit is its motif's count times its number of edges."""
    g = make()
    per_e = E.edge_orbits4_esu(g.n, g.src, g.dst).astype(np.int64)
    per_v = V.orbits4_esu(g.n, g.src, g.dst).astype(np.int64)
    edges = E.edge_list(g.n, g.src, g.dst)
    at_vertex = np.zeros((g.n, len(E.EDGE_ORBITS)), np.int64)
    for k, (a, b) in enumerate(edges):
        at_vertex[a] += per_e[k]
        at_vertex[b] += per_e[k]
    assert np.array_equal(at_vertex, per_v @ INCIDENT)
    glob = O.count4_esu(g.n, g.src, g.dst)
    sums = per_e.sum(axis=0)
    for o in range(len(E.EDGE_ORBITS)):
        assert int(sums[o]) == int(glob[E.EDGE_ORBIT_MOTIF[o]]) * E.EDGE_ORBIT_SIZE[o], E.EDGE_ORBITS[o]


def test_edgeless_and_bad_ids():
    e = np.zeros(0, np.int32)
    assert E.edge_orbits4_esu(6, e, e).shape == (0, 10)
    with pytest.raises(ValueError):
        E.edge_orbits4_brute(3, np.array([0], np.int32), np.array([5], np.int32))


def test_edge_containment_is_unit_upper_triangular():
    M = E.EDGE_CONTAINMENT
    assert M.shape == (10, 10)
    assert np.array_equal(np.diag(M), np.ones(10, np.int64))
    assert not np.tril(M, -1).any()


def test_edge_containment_columns_from_the_motif_graphs():
    """Each motif graph alone: each edge's non-induced statistics are the column of its class."""
    for name, roles in MOTIF_GRAPHS.items():
        s = np.array([a for a, _ in roles], np.int32)
        d = np.array([b for _, b in roles], np.int32)
        N = E.noninduced_per_edge(4, s, d)
        for k, e in enumerate(E.edge_list(4, s, d)):
            assert N[k].tolist() == E.EDGE_CONTAINMENT[:, IDX[roles[e]]].tolist(), (name, e, roles[e])


@pytest.mark.parametrize("seed", range(10))
def test_per_edge_closure_equals_the_definition(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(6, 15))
    p = float(rng.uniform(0.1, 0.85))
    pairs = [(x, y) for x in range(n) for y in range(x + 1, n) if rng.random() < p]
    s = np.array([x for x, _ in pairs], np.int32)
    d = np.array([y for _, y in pairs], np.int32)
    assert np.array_equal(E.edge_orbits4_combo(n, s, d), E.edge_orbits4_brute(n, s, d))


@pytest.mark.parametrize("name,make", [("ba", lambda: graphgen.ba(150, 4, 5)), ("rgg", lambda: graphgen.rgg(150, 7.0, 6)),
                                       ("rmat", lambda: graphgen.rmat(7, 8, seed=4))])
def test_per_edge_closure_on_larger_graphs(name, make):
    g = make()
    assert np.array_equal(E.edge_orbits4_combo(g.n, g.src, g.dst), E.edge_orbits4_esu(g.n, g.src, g.dst))
