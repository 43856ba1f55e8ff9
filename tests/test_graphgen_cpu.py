"""Seeded input generators (no method arithmetic): the induced-subgraph generator of the partitioned
workload's oracle check is exactly the subgraph of the full Chung-Lu graph on the chosen vertices."""
import numpy as np

import graphgen


def _filtered(g, sub):
    pos = -np.ones(g.n, np.int64)
    pos[sub] = np.arange(sub.size)
    keep = (pos[g.src] >= 0) & (pos[g.dst] >= 0)
    return np.sort(pos[g.src[keep]] * sub.size + pos[g.dst[keep]])


def test_chung_lu_induced_equals_the_filtered_full_graph():
    for n, max_w, k, seed, subset_seed in ((200_000, 2000, 30_000, 7, 5), (1_100_000, 4000, 60_000, 3, 9)):
        g = graphgen.chung_lu(n, 2.1, max_w, 10, seed)   # n >= 1e6 takes the threaded chunked path
        sub = graphgen.uniform_subset(n, k, subset_seed)
        h = graphgen.chung_lu_induced(n, 2.1, max_w, 10, seed, sub)
        assert h.n == k
        got = np.sort(h.src.astype(np.int64) * k + h.dst)
        assert np.array_equal(got, _filtered(g, sub)), (n, k)


def test_uniform_subset_is_seeded_distinct_and_sorted():
    a = graphgen.uniform_subset(1_000_000, 5000, 11)
    assert a.size == 5000 and np.all(np.diff(a) > 0) and a[0] >= 0 and a[-1] < 1_000_000
    assert np.array_equal(a, graphgen.uniform_subset(1_000_000, 5000, 11))
    assert not np.array_equal(a, graphgen.uniform_subset(1_000_000, 5000, 12))
    # roughly uniform: each tenth of the id range holds about a tenth of the subset
    counts = np.bincount(a // 100_000, minlength=10)
    assert counts.min() > 400 and counts.max() < 600
