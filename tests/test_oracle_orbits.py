"""Pins of the per-vertex (orbit) oracle: brute force over every 4-subset, closed forms, and the global
counts of the independent C oracle."""
import math
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle as O
from oracle import orbits as R

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import complete, cycle, kbip, path, star, wheel  # noqa: E402

C = math.comb
IDX = {name: i for i, name in enumerate(R.ORBITS)}


def expect(n, per_vertex):
    """Array [n, 11] from {vertex: {orbit name: count}} (missing entries are zero)."""
    out = np.zeros((n, len(R.ORBITS)), np.uint64)
    for v, d in per_vertex.items():
        for name, c in d.items():
            out[v, IDX[name]] = c
    return out


def test_orbit_table_is_consistent():
    # orbit sizes add up to the motif's four vertices
    for motif in range(6):
        assert sum(s for o, s in zip(R.ORBIT_MOTIF, R.ORBIT_SIZE) if o == motif) == 4


@pytest.mark.parametrize("seed", range(12))
def test_esu_equals_brute_force_on_random_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 13))
    p = float(rng.uniform(0.15, 0.8))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    s = np.array([a for a, _ in pairs], np.int32)
    d = np.array([b for _, b in pairs], np.int32)
    assert np.array_equal(R.orbits4_esu(n, s, d), R.orbits4_brute(n, s, d))


@pytest.mark.parametrize("n", [4, 5, 7])
def test_complete_graph(n):
    s, d = complete(n)
    want = expect(n, {v: {"clique": C(n - 1, 3)} for v in range(n)})
    for f in (R.orbits4_brute, R.orbits4_esu):
        assert np.array_equal(f(n, s, d), want)


@pytest.mark.parametrize("k", [3, 4, 6])
def test_star(k):
    s, d = star(k)
    want = expect(k + 1, {0: {"star_center": C(k, 3)}, **{v: {"star_leaf": C(k - 1, 2)} for v in range(1, k + 1)}})
    for f in (R.orbits4_brute, R.orbits4_esu):
        assert np.array_equal(f(k + 1, s, d), want)


@pytest.mark.parametrize("n", [4, 5, 6, 9])
def test_cycle(n):
    s, d = cycle(n)
    per = {v: ({"cycle": 1} if n == 4 else {"path_end": 2, "path_inner": 2}) for v in range(n)}
    for f in (R.orbits4_brute, R.orbits4_esu):
        assert np.array_equal(f(n, s, d), expect(n, per))


@pytest.mark.parametrize("n", [4, 5, 8])
def test_path(n):
    s, d = path(n)
    per = {}
    for i in range(n):
        ends = (i + 3 <= n - 1) + (i - 3 >= 0)          # i is an end of the 4-paths i..i+3 and i-3..i
        inner = (i >= 1 and i + 2 <= n - 1) + (i >= 2 and i + 1 <= n - 1)
        per[i] = {"path_end": ends, "path_inner": inner}
    for f in (R.orbits4_brute, R.orbits4_esu):
        assert np.array_equal(f(n, s, d), expect(n, per))


@pytest.mark.parametrize("a,b", [(2, 3), (3, 4), (4, 4)])
def test_complete_bipartite(a, b):
    s, d = kbip(a, b)
    per = {}
    for v in range(a + b):
        mine, other = (a, b) if v < a else (b, a)
        # 1 + 3 sets are stars; 2 + 2 sets are 4-cycles
        per[v] = {"star_center": C(other, 3), "star_leaf": other * C(mine - 1, 2), "cycle": (mine - 1) * C(other, 2)}
    for f in (R.orbits4_brute, R.orbits4_esu):
        assert np.array_equal(f(a + b, s, d), expect(a + b, per))


@pytest.mark.parametrize("n", [6, 7, 9])
def test_wheel_hub(n):
    """The hub with three rim vertices: no rim edge is a star (the hub its centre), one a paw (the hub
    its degree-3 vertex), two (three consecutive rim vertices) a diamond (the hub on its spine)."""
    s, d = wheel(n)
    got = R.orbits4_esu(n + 1, s, d)
    assert np.array_equal(got, R.orbits4_brute(n + 1, s, d))
    independent = n * C(n - 3, 3) // (n - 3)   # 3-subsets of the n-cycle with no two adjacent
    hub = got[n]
    assert hub[IDX["star_center"]] == independent
    assert hub[IDX["diamond_spine"]] == n
    assert hub[IDX["paw_hub"]] == C(n, 3) - independent - n
    assert hub.sum() == C(n, 3)


@pytest.mark.parametrize("name,make", [("ba", lambda: graphgen.ba(120, 3, 2)), ("er", lambda: graphgen.er(90, 5.0, 3)),
                                       ("rgg", lambda: graphgen.rgg(120, 6.0, 4))])
def test_orbit_sums_are_the_global_counts(name, make):
    """Summed over vertices, each orbit is its motif's count (the C oracle's ESU) times its size."""
    g = make()
    per = R.orbits4_esu(g.n, g.src, g.dst)
    glob = O.count4_esu(g.n, g.src, g.dst)
    sums = per.sum(axis=0)
    for o in range(len(R.ORBITS)):
        assert int(sums[o]) == int(glob[R.ORBIT_MOTIF[o]]) * R.ORBIT_SIZE[o], R.ORBITS[o]


def test_isolated_and_small_inputs():
    e = np.zeros(0, np.int32)
    for n in (0, 1, 3, 6):
        assert R.orbits4_esu(n, e, e).shape == (n, 11) and not R.orbits4_esu(n, e, e).any()
    with pytest.raises(ValueError):
        R.orbits4_esu(3, np.array([0], np.int32), np.array([3], np.int32))


# each motif graph on its own: one occurrence, every vertex's role read off the drawing
MOTIF_GRAPHS = {
    "star": ([(0, 1), (0, 2), (0, 3)], {0: "star_center", 1: "star_leaf", 2: "star_leaf", 3: "star_leaf"}),
    "path": ([(0, 1), (1, 2), (2, 3)], {0: "path_end", 1: "path_inner", 2: "path_inner", 3: "path_end"}),
    "paw": ([(0, 1), (1, 2), (0, 2), (0, 3)], {0: "paw_hub", 1: "paw_side", 2: "paw_side", 3: "paw_pendant"}),
    "cycle": ([(0, 1), (1, 2), (2, 3), (3, 0)], {v: "cycle" for v in range(4)}),
    "diamond": ([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)],
                {0: "diamond_spine", 1: "diamond_spine", 2: "diamond_tip", 3: "diamond_tip"}),
    "clique": ([(a, b) for a in range(4) for b in range(a + 1, 4)], {v: "clique" for v in range(4)}),
}


@pytest.mark.parametrize("name", sorted(MOTIF_GRAPHS))
def test_each_motif_graph_alone(name):
    pairs, roles = MOTIF_GRAPHS[name]
    # relabel by a fixed permutation so the roles do not follow vertex order
    perm = [2, 0, 3, 1]
    s = np.array([perm[a] for a, _ in pairs], np.int32)
    d = np.array([perm[b] for _, b in pairs], np.int32)
    want = expect(4, {perm[v]: {r: 1} for v, r in roles.items()})
    for f in (R.orbits4_brute, R.orbits4_esu):
        assert np.array_equal(f(4, s, d), want)


def test_containment_system_is_unit_upper_triangular():
    M = R.CONTAINMENT
    assert M.shape == (11, 11)
    assert np.array_equal(np.diag(M), np.ones(11, np.int64))
    assert not np.tril(M, -1).any()


@pytest.mark.parametrize("seed", range(10))
def test_per_vertex_closure_equals_the_definition(seed):
    """Eleven non-induced statistics per vertex and the containment inversion give every orbit count
    exactly (random graphs of varied density, including isolated vertices and pendant paths)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 16))
    p = float(rng.uniform(0.1, 0.85))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    s = np.array([a for a, _ in pairs], np.int32)
    d = np.array([b for _, b in pairs], np.int32)
    assert np.array_equal(R.orbits4_combo(n, s, d), R.orbits4_brute(n, s, d))


@pytest.mark.parametrize("name,make", [("ba", lambda: graphgen.ba(150, 4, 5)), ("rgg", lambda: graphgen.rgg(150, 7.0, 6)),
                                       ("rmat", lambda: graphgen.rmat(7, 8, seed=4))])
def test_per_vertex_closure_on_larger_graphs(name, make):
    g = make()
    assert np.array_equal(R.orbits4_combo(g.n, g.src, g.dst), R.orbits4_esu(g.n, g.src, g.dst))


def test_containment_rows_from_the_motif_graphs():
    """Each motif graph alone: the non-induced statistics of each vertex are the containment column
    of its role (the matrix read off the six drawings, independently of the inversion)."""
    for name, (pairs, roles) in MOTIF_GRAPHS.items():
        s = np.array([a for a, _ in pairs], np.int32)
        d = np.array([b for _, b in pairs], np.int32)
        N = R.noninduced_per_vertex(4, s, d)
        for v, role in roles.items():
            assert N[v].tolist() == R.CONTAINMENT[:, IDX[role]].tolist(), (name, v, role)
