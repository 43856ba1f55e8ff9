"""GPU parity of the literal basis (HARP_BASIS_LITERAL: the closure equations of Section III-F as
printed, with the signature cache of Section III-C) against the oracle, bit-exact uint64.

* closed forms (cliques, stars, cycles, paths, complete bipartite graphs, wheels, cocktail parties,
  book graphs whose spine has more common neighbours than a warp stages);
* random graphs against brute force and oracle.count4_literal;
* BA-2000 against oracle.count4_literal, R-MAT scales 14-16 against the stored counts of
  oracle.count4_literal (tests/golden/rmat_literal_oracle.json) and the live oracle.count4_combo;
* both bases forced on the same graphs give identical counts and statistics;
* the signature cache on, off, tiny (most insertions fail) and restricted to a degree bin gives
  identical counts, and its hit rate lies strictly between 0 and 1 on graphs with repeated frontiers;
* harp_select_anchors picks the literal basis on a small graph and the triangle-wedge basis on a
  skewed one, and on both the basis it picks is the faster one measured.
"""
import json
import math
import os
import sys
import time

import numpy as np
import pytest

import graphgen
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import closed_forms, complete, cocktail, edges_of, kbip, star, wheel, cycle  # noqa: E402

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
C = math.comb


@pytest.fixture(scope="module")
def harp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_12074_gb300 import _build, harp as H
    _build.build()
    H.lib()
    return H


def plan_of(H, basis, flags=0, cache_log2=0, min_deg=0):
    p = H.harp_plan()
    p.version = H.HARP_ABI_VERSION
    p.basis = basis
    p.flags = flags
    p.lit_cache_log2 = cache_log2
    p.lit_cache_min_deg = min_deg
    return p


def lit_count(H, n, src, dst, **kw):
    g = H.harp_build_csr(n, torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda())
    try:
        counts, stats = H.harp_count4_stats(g, plan_of(H, H.HARP_BASIS_LITERAL, **kw))
        reuse = H.harp_reuse_stats(g)
    finally:
        g.close()
    return counts, stats, reuse


def book(k):
    """Spine 0 - 1 and k pages adjacent to both: 2 C(k,3) stars (one per spine vertex), C(k,2) diamonds."""
    return edges_of([(0, 1)] + [(0, 2 + i) for i in range(k)] + [(1, 2 + i) for i in range(k)])


LIT_CLOSED = closed_forms(scale=1) + [
    ("K40", 40, complete(40), [0, 0, 0, 0, 0, C(40, 4)]),
    ("K300", 300, complete(300), [0, 0, 0, 0, 0, C(300, 4)]),
    ("K1,5000", 5001, star(5000), [C(5000, 3), 0, 0, 0, 0, 0]),
    ("W5000", 5001, wheel(5000), [5000 * C(4997, 3) // 4997, 5000, 5000 * 4996, 0, 5000, 0]),
    ("K40,60", 100, kbip(40, 60), [40 * C(60, 3) + 60 * C(40, 3), 0, 0, C(40, 2) * C(60, 2), 0, 0]),
    ("K300,500", 800, kbip(300, 500), [300 * C(500, 3) + 500 * C(300, 3), 0, 0, C(300, 2) * C(500, 2), 0, 0]),
    ("CP40", 80, cocktail(40), [0, 0, 0, C(40, 2), 4 * 40 * C(39, 2), 16 * C(40, 4)]),
    ("C100000", 100000, cycle(100000), [0, 100000, 0, 0, 0, 0]),
    ("book40", 42, book(40), [2 * C(40, 3), 0, 0, 0, C(40, 2), 0]),
    ("book600", 602, book(600), [2 * C(600, 3), 0, 0, 0, C(600, 2), 0]),  # C_01 has 600 > 512 members
]


@pytest.mark.parametrize("name,n,e,want", LIT_CLOSED, ids=[c[0] for c in LIT_CLOSED])
def test_literal_closed_forms(harp, name, n, e, want):
    s, d = e
    counts, _, _ = lit_count(harp, n, s, d)
    assert counts.tolist() == [w % 2**64 for w in want]


def test_book_graph_closed_form_against_brute_force():
    """The book graph's closed form itself, checked by brute force on a small page count."""
    s, d = book(7)
    assert O.count4_brute(9, s, d).tolist() == [2 * C(7, 3), 0, 0, 0, C(7, 2), 0]


def test_literal_random_graphs_against_brute_force_and_literal_oracle(harp):
    rng = np.random.default_rng(2024)
    for trial in range(40):
        n = int(rng.integers(5, 40))
        p = float(rng.uniform(0.05, 0.6))
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.size) < p
        s, d = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
        want = O.count4_brute(n, s, d).tolist()
        assert O.count4_literal(n, s, d).tolist() == want
        counts, _, _ = lit_count(harp, n, s, d)
        assert counts.tolist() == want, (trial, n, p)


def test_literal_ba2000_against_literal_oracle(harp):
    g = graphgen.ba_2000()
    counts, _, _ = lit_count(harp, g.n, g.src, g.dst)
    assert counts.tolist() == O.count4_literal(g.n, g.src, g.dst).tolist()


@pytest.mark.parametrize("scale", [14, 15, 16])
def test_literal_rmat_against_stored_literal_oracle(harp, scale):
    with open(os.path.join(HERE, "golden", "rmat_literal_oracle.json")) as f:
        rec = json.load(f)[str(scale)]
    g = graphgen.rmat(scale, 16, 0.57, 0.19, 0.19, seed=1)
    assert rec["graph"] == g.name
    counts, _, _ = lit_count(harp, g.n, g.src, g.dst)
    assert counts.tolist() == rec["literal"]
    assert counts.tolist() == O.count4_combo(g.n, g.src, g.dst).tolist()


def test_both_bases_give_identical_counts_and_statistics(harp):
    graphs = [graphgen.er(3000, 12.0, 3), graphgen.rgg(4000, 14.0, 5), graphgen.ba(5000, 6, 7),
              graphgen.rmat(13, 16, 0.57, 0.19, 0.19, seed=9), graphgen.chung_lu(20000, 2.1, 800, 8, 4)]
    for g in graphs:
        csr = harp.harp_build_csr(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
        try:
            tw = harp.harp_count4_stats(csr, plan_of(harp, harp.HARP_BASIS_TRIANGLE_WEDGE))
            lit = harp.harp_count4_stats(csr, plan_of(harp, harp.HARP_BASIS_LITERAL))
        finally:
            csr.close()
        assert tw[0].tolist() == lit[0].tolist(), g.name
        assert tw[1].tolist() == lit[1].tolist(), g.name
        assert tw[0].tolist() == O.count4_combo(g.n, g.src, g.dst).tolist(), g.name


def test_signature_cache_never_changes_counts_and_hits_below_one(harp):
    """Cache on (default size), off, 16 slots (most frontiers find no slot) and admitting only pairs of
    degree >= 8: identical counts.  On graphs whose non-adjacent pairs share several common neighbours
    the same frontier is requested repeatedly, so the default cache hits, yet below every request.
    (Admitting only the higher degree bin can raise the hits: the low-degree frontiers it leaves out
    no longer take the slots of the probe windows.)"""
    for g in (graphgen.ba(3000, 5, 11), graphgen.rgg(3000, 10.0, 12), graphgen.rmat(12, 16, seed=13)):
        want = O.count4_combo(g.n, g.src, g.dst).tolist()
        counts, _, (lookups, hits) = lit_count(harp, g.n, g.src, g.dst)
        assert counts.tolist() == want, g.name
        assert 0 < hits < lookups, (g.name, lookups, hits)
        for kw in ({"flags": harp.HARP_PLAN_NO_REUSE}, {"cache_log2": 4}, {"min_deg": 8}):
            c2, _, (lk2, ht2) = lit_count(harp, g.n, g.src, g.dst, **kw)
            assert c2.tolist() == want, (g.name, kw)
            if "flags" in kw:
                assert ht2 == 0
            elif "cache_log2" in kw:
                assert ht2 < hits, (g.name, kw)
            else:  # admission by degree bin: fewer candidates, less pressure on the probe windows
                assert 0 < ht2 < lk2, (g.name, kw)
    # K_{300,500}: the 44,850 non-adjacent pairs of the 300 side have the 500 side as common frontier,
    # requested about a thousand times each (once per edge scan that meets them).  The first requests
    # of a pair all miss while the warps that made them compute it (one warp per out-arc, ~15 arcs a
    # warp here; on a graph with fewer arcs than warps every request is such a first one), the rest
    # hit.
    s, d = kbip(300, 500)
    counts, _, (lookups, hits) = lit_count(harp, 800, s, d)
    assert counts.tolist() == [300 * C(500, 3) + 500 * C(300, 3), 0, 0, C(300, 2) * C(500, 2), 0, 0]
    assert 0.5 < hits / lookups < 1.0, (lookups, hits)


def _median_ms(H, csr, plan, reps=15):
    H.harp_count4(csr, plan)
    ts = []
    for _ in range(reps):
        t = time.perf_counter()
        H.harp_count4(csr, plan)
        ts.append(1000 * (time.perf_counter() - t))
    return float(np.median(ts))


def test_planner_picks_the_faster_basis(harp):
    """Eq. 1 weighs the literal basis's larger enumeration against its fewer launches: on a small
    graph the launches decide (literal), on a skewed one the enumeration (triangle-wedge).  Both
    choices are checked against measured wall time of harp_count4 under each forced basis."""
    cases = [(graphgen.ba(300, 3, 21), "lit"), (graphgen.rmat(16, 16, 0.57, 0.19, 0.19, seed=1), "tw")]
    for g, expect in cases:
        csr = harp.harp_build_csr(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
        try:
            p = harp.harp_select_anchors(csr)
            t_tw = _median_ms(harp, csr, plan_of(harp, harp.HARP_BASIS_TRIANGLE_WEDGE))
            t_lit = _median_ms(harp, csr, plan_of(harp, harp.HARP_BASIS_LITERAL))
            counts = harp.harp_count4(csr, p)
        finally:
            csr.close()
        chosen = "lit" if p.basis == harp.HARP_BASIS_LITERAL else "tw"
        assert chosen == expect, (g.name, p.est_cost_tw, p.est_cost_lit, t_tw, t_lit)
        faster = "lit" if t_lit < t_tw else "tw"
        assert chosen == faster, (g.name, t_tw, t_lit)
        assert counts.tolist() == O.count4_combo(g.n, g.src, g.dst).tolist()
