"""Pins of the 5-vertex motif oracle: the class table against known enumerations, closed forms, each
class graph alone, ESU against brute force."""
import itertools
import math
import os
import sys

import numpy as np
import pytest

from oracle import motifs5 as M

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import complete, cycle, kbip, path, star  # noqa: E402

C = math.comb
STAR4 = M.class_of_edges([(0, 1), (0, 2), (0, 3), (0, 4)])
PATH5 = M.class_of_edges([(0, 1), (1, 2), (2, 3), (3, 4)])
CYCLE5 = M.class_of_edges([(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)])
K5 = M.class_of_edges(list(itertools.combinations(range(5), 2)))
K23 = M.class_of_edges([(a, b) for a in (0, 1) for b in (2, 3, 4)])


def both(n, s, d):
    a, b = M.count5_brute(n, s, d), M.count5_esu(n, s, d)
    assert np.array_equal(a, b)
    return a


def unit(i, c=1):
    out = np.zeros(len(M.CLASSES), np.uint64)
    out[i] = c
    return out


def test_class_table_matches_known_enumerations():
    # 21 connected graphs on five unlabelled vertices; 728 connected labelled graphs on five vertices
    assert len(M.CLASSES) == 21
    connected = [m for m in range(1 << 10) if M._CANON[m] is not None]
    assert len(connected) == 728
    # orbit-stabiliser: each class has 120 / |Aut| labellings
    sizes = {}
    for m in connected:
        sizes[M._CANON[m]] = sizes.get(M._CANON[m], 0) + 1
    for key, size in sizes.items():
        edges = M._edges_of(key)
        aut = sum(1 for p in itertools.permutations(range(5))
                  if M._mask([(p[a], p[b]) for a, b in edges]) == key)
        assert size * aut == 120
    # edge counts of the classes: 4 (trees: 3), 5 (5), 6 (5), 7 (4), 8 (2), 9 (1), 10 (1)
    per_edges = [bin(c).count("1") for c in M.CLASSES]
    assert [per_edges.count(e) for e in range(4, 11)] == [3, 5, 5, 4, 2, 1, 1]


@pytest.mark.parametrize("i", range(21))
def test_each_class_graph_alone(i):
    edges = M.class_edges(i)
    perm = [4, 2, 0, 3, 1]
    s = np.array([perm[a] for a, _ in edges], np.int32)
    d = np.array([perm[b] for _, b in edges], np.int32)
    assert np.array_equal(both(5, s, d), unit(i))


@pytest.mark.parametrize("n", [5, 6, 8])
def test_complete_graph(n):
    s, d = complete(n)
    assert np.array_equal(both(n, s, d), unit(K5, C(n, 5)))


@pytest.mark.parametrize("k", [4, 6])
def test_star(k):
    s, d = star(k)
    assert np.array_equal(both(k + 1, s, d), unit(STAR4, C(k, 4)))


@pytest.mark.parametrize("n", [5, 6, 9])
def test_cycle(n):
    s, d = cycle(n)
    assert np.array_equal(both(n, s, d), unit(CYCLE5, 1) if n == 5 else unit(PATH5, n))


@pytest.mark.parametrize("n", [5, 7, 10])
def test_path(n):
    s, d = path(n)
    assert np.array_equal(both(n, s, d), unit(PATH5, n - 4))


@pytest.mark.parametrize("a,b", [(2, 3), (3, 4), (2, 6)])
def test_complete_bipartite(a, b):
    s, d = kbip(a, b)
    want = unit(STAR4, a * C(b, 4) + b * C(a, 4)) + unit(K23, C(a, 2) * C(b, 3) + C(a, 3) * C(b, 2))
    assert np.array_equal(both(a + b, s, d), want)


@pytest.mark.parametrize("seed", range(8))
def test_esu_equals_brute_force_and_totals(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(6, 12))
    p = float(rng.uniform(0.15, 0.8))
    pairs = [(x, y) for x in range(n) for y in range(x + 1, n) if rng.random() < p]
    s = np.array([x for x, _ in pairs], np.int32)
    d = np.array([y for _, y in pairs], np.int32)
    got = both(n, s, d)
    # total = connected 5-subsets, by a search that does not use the class table
    adj = [set() for _ in range(n)]
    for x, y in pairs:
        adj[x].add(y)
        adj[y].add(x)

    def connected(sub):
        seen, stack = {sub[0]}, [sub[0]]
        while stack:
            for y in adj[stack.pop()] & set(sub):
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
        return len(seen) == 5
    assert int(got.sum()) == sum(1 for sub in itertools.combinations(range(n), 5) if connected(sub))


def test_bad_input():
    with pytest.raises(ValueError):
        M.count5_esu(3, np.array([0], np.int32), np.array([4], np.int32))
    with pytest.raises(ValueError):
        M.class_of_edges([(0, 1), (2, 3)])
