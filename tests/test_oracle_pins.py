"""Pins for the CPU oracle (no GPU).

The oracle is trusted only after it agrees with things it does not compute itself:
closed forms derived from the definition of an induced occurrence (Section II), exact integer
matrix identities (tr A^3, tr A^4), hand-derived fixtures, and brute force over all 4-subsets.
Each check is chosen so that a dropped term, a wrong sign or a transposed operand fails one of them.
"""
import json
import math
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
C = math.comb
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


from graph_families import closed_forms, complete, edges_of, star  # noqa: E402


ALL = ("brute", "esu", "literal", "combo")


def run(method, n, s, d):
    return {"brute": O.count4_brute, "esu": O.count4_esu, "literal": O.count4_literal,
            "combo": O.count4_combo}[method](n, s, d)


CLOSED = closed_forms()


@pytest.mark.parametrize("method", ALL)
@pytest.mark.parametrize("name,n,e,want", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(method, name, n, e, want):
    s, d = e
    assert run(method, n, s, d).tolist() == want


def _fixtures():
    out = []
    with open(os.path.join(GOLDEN, "closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, n, es, counts, _why = [x.strip() for x in line.split("|")]
            pairs = [tuple(map(int, x.split("-"))) for x in es.split()]
            out.append((name, int(n), pairs, [int(x) for x in counts.split()]))
    return out


@pytest.mark.parametrize("method", ALL)
@pytest.mark.parametrize("name,n,pairs,want", _fixtures(), ids=[f[0] for f in _fixtures()])
def test_hand_fixtures(method, name, n, pairs, want):
    s, d = edges_of(pairs)
    assert run(method, n, s, d).tolist() == want


def _golden_random():
    with open(os.path.join(GOLDEN, "brute_random.json")) as f:
        return json.load(f)["graphs"]


@pytest.mark.parametrize("method", ("esu", "literal", "combo"))
def test_stored_brute_force(method):
    for g in _golden_random():
        got = run(method, g["n"], np.array(g["src"], np.int32), np.array(g["dst"], np.int32))
        assert got.tolist() == g["counts"], g["name"]


def _random_graphs(count, nmax, seed0):
    out = []
    for i in range(count):
        n = 5 + (i * 13) % (nmax - 4)
        k = 1.5 + (i * 5) % 11
        gen = (graphgen.er, graphgen.rgg)[i % 2]
        g = gen(n, k, seed0 + i)
        out.append(g)
    for i in range(count // 4):
        out.append(graphgen.ba(12 + i * 3, 1 + i % 4, seed0 + 1000 + i))
    return out


def test_all_methods_agree_with_brute_force():
    for g in _random_graphs(60, 40, 11):
        want = O.count4_brute(g.n, g.src, g.dst)
        for m in ("esu", "literal", "combo"):
            assert run(m, g.n, g.src, g.dst).tolist() == want.tolist(), (m, g.name)


def _dense(n, s, d):
    A = np.zeros((n, n), np.int64)
    for a, b in zip(s.tolist(), d.tolist()):
        if a != b:
            A[a, b] = A[b, a] = 1
    return A


@pytest.mark.parametrize("gen,n,k,seed", [(graphgen.er, 300, 12, 1), (graphgen.rgg, 600, 20, 2),
                                          (graphgen.ba, 800, 6, 3), (graphgen.er, 150, 60, 4)])
def test_noninduced_against_matrix_powers(gen, n, k, seed):
    """tr(A^3) = 6T; tr(A^4) = 8 C4_non + 4 sum_v C(d_v, 2) + 2m; sum_v C(d,3); exact int64."""
    g = gen(n, k, seed)
    A = _dense(g.n, g.src, g.dst)
    A2 = A @ A
    deg = A.sum(1)
    m = int(A.sum()) // 2
    st = O.noninduced(g.n, g.src, g.dst).astype(object)
    T, K4, C4n, Sn, Pn, pawn, Dn, mm = st.tolist()
    assert mm == m
    assert int((A2 * A).sum()) == 6 * T
    tr4 = int((A2 * A2).sum())
    assert tr4 == 8 * C4n + 4 * sum(C(int(x), 2) for x in deg) + 2 * m
    assert Sn == sum(C(int(x), 3) for x in deg)
    # per-edge triangles from A^2 restricted to edges; sum_e C(t_e,2) and sum_e (d_u-1)(d_v-1) - 3T
    iu, ju = np.nonzero(np.triu(A))
    te = A2[iu, ju]
    assert Dn == sum(C(int(t), 2) for t in te)
    assert Pn == int(((deg[iu] - 1) * (deg[ju] - 1)).sum()) - 3 * T
    tv = (A2 * A).sum(1) // 2
    assert pawn == int((tv * np.maximum(deg - 2, 0)).sum())
    # 4-cliques: sum over triangles of common neighbours, each K4 counted 4 times
    A3 = np.einsum("ij,jk,ki->", A, A, A)
    assert A3 == 6 * T


def test_linear_identities_tie_noninduced_to_induced():
    """Non-induced sums = containment matrix x brute-force induced counts (rows: S, P, paw, C4, D)."""
    for g in _random_graphs(30, 30, 77):
        star_, path_, paw, c4, dia, k4 = [int(x) for x in O.count4_brute(g.n, g.src, g.dst)]
        T, K4, C4n, Sn, Pn, pawn, Dn, m = [int(x) for x in O.noninduced(g.n, g.src, g.dst)]
        assert K4 == k4
        assert Dn == dia + 6 * k4
        assert C4n == c4 + dia + 3 * k4
        assert pawn == paw + 4 * dia + 12 * k4
        assert Pn == path_ + 2 * paw + 4 * c4 + 6 * dia + 12 * k4
        assert Sn == star_ + paw + 2 * dia + 4 * k4


def test_edge_triangles_against_matrix():
    g = graphgen.er(200, 25, 9)
    A = _dense(g.n, g.src, g.dst)
    A2 = A @ A
    eu, ev, te = O.edge_triangles(g.n, g.src, g.dst)
    assert np.all(eu < ev)
    assert te.astype(np.int64).tolist() == A2[eu, ev].tolist()
    assert len(eu) == int(A.sum()) // 2


def test_invariances():
    rng = np.random.default_rng(5)
    for g in _random_graphs(8, 60, 300):
        want = O.count4_esu(g.n, g.src, g.dst)
        perm = rng.permutation(g.n).astype(np.int32)
        s2, d2 = perm[g.src], perm[g.dst]
        assert O.count4_esu(g.n, s2, d2).tolist() == want.tolist()
        # duplicates, reversed copies, self-loops, shuffled order
        s3 = np.concatenate([g.src, g.dst, g.src[:3], np.arange(min(4, g.n), dtype=np.int32)])
        d3 = np.concatenate([g.dst, g.src, g.dst[:3], np.arange(min(4, g.n), dtype=np.int32)])
        o = rng.permutation(len(s3))
        assert O.count4_combo(g.n, s3[o], d3[o]).tolist() == want.tolist()
        # isolated extra vertices change nothing
        assert O.count4_combo(g.n + 7, g.src, g.dst).tolist() == want.tolist()


def test_plain_workload_methods_agree():
    """Barabasi-Albert n=2000, m=4, seed 1: ESU, literal closure and inversion agree."""
    g = graphgen.ba_2000()
    a = O.count4_esu(g.n, g.src, g.dst)
    assert O.count4_literal(g.n, g.src, g.dst).tolist() == a.tolist()
    assert O.count4_combo(g.n, g.src, g.dst).tolist() == a.tolist()
    m, _ = O.graph_summary(g.n, g.src, g.dst)
    assert m == 7990


def test_modular_binomials_large_degree():
    """S_non for a star with 3,000,000 leaves: C(d,3) is exact modulo 2^64 (divisions taken first)."""
    k = 3_000_000
    s, d = star(k)
    st = O.noninduced(k + 1, s, d)
    assert int(st[3]) == C(k, 3) % 2**64
    assert O.count4_combo(k + 1, s, d).tolist() == [C(k, 3) % 2**64, 0, 0, 0, 0, 0]


def test_invalid_ids_rejected():
    with pytest.raises(ValueError):
        O.count4_esu(3, np.array([0, 5], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(ValueError):
        O.count4_combo(3, np.array([-1], np.int32), np.array([1], np.int32))


def test_empty_and_degenerate():
    e = np.zeros(0, np.int32)
    for m in ALL:
        assert run(m, 0, e, e).tolist() == [0] * 6
        assert run(m, 3, e, e).tolist() == [0] * 6
    s, d = complete(3)
    for m in ALL:
        assert run(m, 3, s, d).tolist() == [0] * 6
