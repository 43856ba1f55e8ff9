"""Owner-rule partitioned counting (GPU): every partition count k gives exactly the counts of the
unpartitioned path and of the oracle, whether the ranges are forced (k in {1, 2, 3, 7, 16}) or sized to
a small device budget."""
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import cocktail, complete, kbip, wheel  # noqa: E402

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


def graphs():
    out = [graphgen.ba_2000(), graphgen.er(3000, 40, 5), graphgen.rgg(5000, 20, 6), graphgen.rmat(14, 16, seed=2),
           graphgen.chung_lu(20000, 2.1, 1500, 12, 7)]
    for name, (n, e) in {"K300": (300, complete(300)), "W3000": (3001, wheel(3000)),
                         "K120,200": (320, kbip(120, 200)), "CP80": (160, cocktail(80))}.items():
        out.append(graphgen.Graph(n, e[0], e[1], name))
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 7, 16])
def test_forced_partitions_match_whole_graph(harp, k):
    for g in graphs():
        whole = harp.count4_edges(g.n, g.src, g.dst)
        got, st = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=1 << 34, parts=k)
        assert got.tolist() == whole.tolist(), (g.name, k)
        assert st["partitions"] == 2 * k               # k triangle ranges and k wedge ranges


@pytest.mark.parametrize("make", [lambda: graphgen.rmat(15, 16, seed=4), lambda: graphgen.rgg(40000, 16, 9),
                                  lambda: graphgen.er(30000, 12, 3)])
def test_budget_sized_partitions_and_oracle(harp, make):
    g = make()
    want = O.count4_combo(g.n, g.src, g.dst)
    whole, st1 = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=1 << 34)
    assert st1["partitions"] == 2                      # one triangle block, one wedge block
    # the largest range of 16 equal ranges fits any range the greedy cut can start (its halo contains
    # the halo of every single vertex of that range); below the whole graph's footprint it must cut
    _, st16 = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=1 << 34, parts=16)
    budget = st16["device_peak_bytes"]
    got, st = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=budget)
    if budget < st1["device_peak_bytes"]:
        assert st["partitions"] > 2
    assert st["device_peak_bytes"] <= budget
    assert got.tolist() == whole.tolist() == want.tolist()
    with pytest.raises(harp.HarpError) as ei:    # below every single-vertex halo of the top range
        harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=st16["device_peak_bytes"] // 64)
    assert ei.value.status == harp.HARP_ENOMEM


def test_partitioned_errors(harp):
    with pytest.raises(harp.HarpError) as ei:
        harp.harp_count4_partitioned(4, [0, 9], [1, 2], budget_bytes=1 << 30)
    assert ei.value.status == harp.HARP_EINVAL
    g = graphgen.er(2000, 10, 1)
    with pytest.raises(harp.HarpError) as ei:
        harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=1024)  # the per-vertex arrays alone exceed it
    assert ei.value.status == harp.HARP_ENOMEM


def test_chung_lu_large_induced_subsample_under_a_cap(harp):
    """The partitioned large graph's oracle check: the subgraph of the 5e7-vertex Chung-Lu workload
    (exponent 2.1, max expected degree 1e6, mean degree 48, seed 1) induced on a seeded uniform
    1e6-vertex subset, counted the same way as the whole workload (budget-sized triangle ranges and
    wedge blocks, here below the subsample's own footprint so that it is cut), against the oracle.
    (Scaling the 24 GiB cap by the subsample's share of the edges would put the budget below its
    per-vertex arrays alone; the budget is instead set between the one-block and the 16-range
    footprints, which forces several blocks.)"""
    g = graphgen.chung_lu_large_induced()
    assert g.n == 1_000_000 and g.m_in > 300_000
    want = O.count4_combo(g.n, g.src, g.dst)
    whole, st1 = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=1 << 34)
    _, st16 = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=1 << 34, parts=16)
    budget = (st1["device_peak_bytes"] + st16["device_peak_bytes"]) // 2
    got, st = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=budget)
    assert st["partitions"] > 2 and st["device_peak_bytes"] <= budget
    assert st["transfer_ms"] >= 0 and st["device_ms"] > 0
    assert got.tolist() == whole.tolist() == want.tolist()
    assert harp.count4_edges(g.n, g.src, g.dst).tolist() == want.tolist()


def test_wedge_blocks_cut_into_x_slices(harp):
    """A budget that holds the roots' lists but not the rows of their lower neighbours forces the
    wedge blocks of a hub-heavy graph into x-slices; the counts stay exact."""
    g = graphgen.chung_lu(60000, 2.1, 3000, 16, 21)
    want = O.count4_combo(g.n, g.src, g.dst)
    whole, st1 = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=1 << 34)
    assert st1["wedge_sliced"] == 0 and st1["tri_blocks"] == 1 and st1["wedge_blocks"] == 1
    lo, hi = 0, st1["device_peak_bytes"]
    got = None
    for _ in range(24):  # the largest budget below the whole footprint that slices
        mid = (lo + hi) // 2
        try:
            c, st = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=mid)
        except harp.HarpError as e:
            assert e.status == harp.HARP_ENOMEM
            lo = mid
            continue
        if st["wedge_sliced"] > 0:
            got = (c, st)
            break
        hi = mid
    assert got is not None, "no budget produced x-sliced wedge blocks"
    c, st = got
    assert st["wedge_blocks"] == st["partitions"] - st["tri_blocks"] and st["device_peak_bytes"] <= mid
    assert c.tolist() == whole.tolist() == want.tolist()
