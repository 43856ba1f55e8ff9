"""Induced-signature reuse (Section III-C) on the GPU: switching reuse off, shrinking the staged
capacity, narrowing the warp mode or changing the membership probe changes the work, never the
counts; the hit counters account for every 4-clique extension (one lookup per triangle)."""
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import cocktail, complete, wheel  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def harp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_12074_gb300 import _build, harp as H
    _build.build()
    H.lib()
    return H


def hub_fan(nb=1030, nc=1100):
    """Anchors whose out-degree exceeds the shared-memory stage: vertex a and every c in C have the
    nb vertices of B (degree nc + 1 or more) as out-neighbours, and a path through B closes
    triangles (a, b_i, b_i+1) and (c, b_i, b_i+1): global-staged by default, unstaged fallback when
    tri_big_max forbids that stage.  A disjoint K40 adds shared-memory-staged anchors."""
    a, B, C = 0, np.arange(1, 1 + nb), np.arange(1 + nb, 1 + nb + nc)
    k_src, k_dst = complete(40)
    base = 1 + nb + nc
    src = [np.full(nb, a), np.repeat(B, nc), B[:-1], np.asarray(k_src) + base]
    dst = [B, np.tile(C, nb), B[1:], np.asarray(k_dst) + base]
    return graphgen.Graph(base + 40, np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32),
                          "HUBFAN")


def graphs():
    out = [graphgen.ba_2000(), graphgen.rmat(14, 16, seed=5), graphgen.er(3000, 30, 2),
           graphgen.chung_lu(20000, 2.1, 2000, 16, 3), hub_fan()]
    for name, (n, e) in {"K40": (40, complete(40)), "K300": (300, complete(300)),
                         "W3000": (3001, wheel(3000)), "CP200": (400, cocktail(200))}.items():
        out.append(graphgen.Graph(n, e[0], e[1], name))
    return out


def plan(H, **kw):
    p = H.harp_plan()
    p.version = H.HARP_ABI_VERSION
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def run(H, g, p=None):
    c = H.harp_build_csr(g.n, g.src, g.dst)
    try:
        counts, stats = H.harp_count4_stats(c, p)
        look, hits = H.harp_reuse_stats(c)
        return counts.tolist(), stats.tolist(), look, hits
    finally:
        c.close()


def test_reuse_switch_and_capacity_never_change_counts(harp):
    H = harp
    variants = {
        "no_reuse": plan(H, flags=H.HARP_PLAN_NO_REUSE),
        "cta256": plan(H, tri_cta_max=256),
        "cta1": plan(H, tri_cta_max=1),                       # above the warp mode: global-staged
        "nobig": plan(H, tri_big_max=1),                      # above the CTA mode: unstaged fallback
        "cta1_nobig": plan(H, tri_cta_max=1, tri_big_max=1),  # every anchor above the warp mode unstaged
        "warp8": plan(H, tri_warp_max=8),
        "bsearch": plan(H, tri_probe=H.HARP_PROBE_BSEARCH),
        "bsearch_no_reuse": plan(H, tri_probe=H.HARP_PROBE_BSEARCH, flags=H.HARP_PLAN_NO_REUSE),
    }
    for g in graphs():
        counts, stats, look, hits = run(H, g)
        assert look == stats[0], g.name                      # one lookup per triangle
        assert hits <= look
        if g.name in ("K40", "K300", "CP200", "W3000", "HUBFAN"):
            assert hits == look                              # everything staged (shared or global)
        for name, p in variants.items():
            c2, s2, l2, h2 = run(H, g, p)
            assert c2 == counts and s2 == stats, (g.name, name)
            assert l2 == look
            if "no_reuse" in name:
                assert h2 == 0, (g.name, name)
            elif "nobig" in name:
                assert h2 <= hits, (g.name, name)
                if g.name == "HUBFAN":                       # out-degree 1030 unstaged: misses
                    assert 0 < h2 < look
            else:                                            # same staging, other tier split or probe
                assert h2 == hits, (g.name, name)


def test_reuse_counts_against_oracle(harp):
    H = harp
    g = graphgen.chung_lu(8000, 2.1, 1500, 12, 11)
    want = O.count4_combo(g.n, g.src, g.dst).tolist()
    for p in (None, plan(H, flags=H.HARP_PLAN_NO_REUSE), plan(H, tri_cta_max=1),
              plan(H, tri_cta_max=1, flags=H.HARP_PLAN_NO_REUSE), plan(H, tri_cta_max=1, tri_big_max=1)):
        assert run(H, g, p)[0] == want


def test_reuse_stats_before_count(harp):
    H = harp
    g = graphgen.ba(200, 3, 1)
    c = H.harp_build_csr(g.n, g.src, g.dst)
    try:
        with pytest.raises(H.HarpError) as ei:
            H.harp_reuse_stats(c)
        assert ei.value.status == H.HARP_ENOTFOUND
    finally:
        c.close()


def test_batch_without_reuse(harp):
    H = harp
    gs = [graphgen.batch_graph(s, n_lo=50, n_hi=3000) for s in range(40)] + [
        graphgen.Graph(300, *complete(300), "K300")]
    cs = [H.harp_build_csr(g.n, g.src, g.dst) for g in gs]
    try:
        a = H.harp_count4_batch(cs)
        b = H.harp_count4_batch(cs, plan(H, flags=H.HARP_PLAN_NO_REUSE | H.HARP_PLAN_NO_GRAPH))
        c = H.harp_count4_batch(cs, plan(H, tri_cta_max=64, tri_warp_max=4))
        assert a.tolist() == b.tolist() == c.tolist()
    finally:
        for c_ in cs:
            c_.close()
