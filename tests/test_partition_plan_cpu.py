"""The partition planner (harp_partition_plan) on the host: no device is needed when a budget is given.

The planner cuts the rank-ordered graph exactly as the partitioned count does: triangle anchors by
rank ranges of their lowest vertex, wedge anchors by rank ranges of their top vertex, each cut into
slices of the opposite vertex x.  An anchor belongs to exactly one block only if the ranges tile the
rank space and, per root range, the x-slices tile it too; and every block must fit the budget.
"""
import numpy as np
import pytest

import graphgen

H = pytest.importorskip("paper_2607_12074_gb300.harp")

GRAPHS = {
    "ba5000": lambda: graphgen.ba(5000, 4, 3),
    "chung_lu50k": lambda: graphgen.chung_lu(50_000, 2.1, 2000, 6, 7),
    "rmat14": lambda: graphgen.rmat(14, 16, seed=5),
}


@pytest.fixture(scope="module")
def lib():
    H.lib()
    return H


def check_tiling(n, tri, wedge):
    """Triangle ranges tile [0, n); wedge root ranges tile [0, n) and each one's x-slices tile [0, n)."""
    assert tri[0, 0] == 0 and tri[-1, 1] == n
    assert np.all(tri[1:, 0] == tri[:-1, 1]) and np.all(tri[:, 0] < tri[:, 1])
    ranges = []
    for lo, hi, xlo, xhi in wedge.tolist():
        if not ranges or ranges[-1][:2] != (lo, hi):
            ranges.append((lo, hi, []))
        ranges[-1][2].append((xlo, xhi))
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (lo0, hi0, _), (lo1, hi1, _) in zip(ranges, ranges[1:]):
        assert hi0 == lo1 and lo1 < hi1
    for lo, hi, slices in ranges:
        assert slices[0][0] == 0 and slices[-1][1] == n, (lo, hi, slices[:3])
        assert all(a[1] == b[0] for a, b in zip(slices, slices[1:])), (lo, hi)
        assert all(a < b for a, b in slices)
    return ranges


def smallest_feasible_budget(lib, g, hi):
    """Bisection for the smallest budget the planner accepts (feasibility grows with the budget)."""
    lo = 1
    while hi - lo > max(1, hi >> 12):
        mid = (lo + hi) // 2
        try:
            lib.harp_partition_plan(g.n, g.src, g.dst, mid)
            hi = mid
        except lib.HarpError as e:
            assert e.status == lib.HARP_ENOMEM
            lo = mid
    return hi


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_budget_sized_blocks_tile_and_fit(lib, name):
    g = GRAPHS[name]()
    whole, tri, wedge = lib.harp_partition_plan(g.n, g.src, g.dst, 1 << 40)
    assert (whole["tri_blocks"], whole["wedge_blocks"], whole["wedge_sliced"]) == (1, 1, 0)
    assert tri.tolist() == [[0, g.n]] and wedge.tolist() == [[0, g.n, 0, g.n]]
    assert whole["device_ms"] == 0 and whole["h2d_bytes"] == 0
    peak = whole["device_peak_bytes"]
    low = smallest_feasible_budget(lib, g, peak)
    most = 0
    for budget in sorted({low, (low + peak) // 2, (3 * low + peak) // 4, peak}):
        st, tri, wedge = lib.harp_partition_plan(g.n, g.src, g.dst, budget)
        assert st["device_peak_bytes"] <= budget
        assert st["partitions"] == st["tri_blocks"] + st["wedge_blocks"]
        assert st["m"] == whole["m"]
        ranges = check_tiling(g.n, tri, wedge)
        assert st["wedge_sliced"] == sum(len(r[2]) for r in ranges if len(r[2]) > 1)
        most = max(most, st["partitions"])
    assert most > 2  # the tightest budget splits the graph


@pytest.mark.parametrize("parts", [1, 2, 3, 7])
def test_forced_parts_are_equal_rank_ranges(lib, parts):
    g = graphgen.ba(3000, 3, 1)
    st, tri, wedge = lib.harp_partition_plan(g.n, g.src, g.dst, 1 << 40, parts)
    want = [[g.n * k // parts, g.n * (k + 1) // parts] for k in range(parts)]
    assert tri.tolist() == want
    assert wedge.tolist() == [r + [0, g.n] for r in want]
    assert (st["tri_blocks"], st["wedge_blocks"], st["wedge_sliced"]) == (parts, parts, 0)


def test_tighter_budgets_never_take_fewer_blocks(lib):
    g = graphgen.chung_lu(50_000, 2.1, 2000, 6, 7)
    peak = lib.harp_partition_plan(g.n, g.src, g.dst, 1 << 40)[0]["device_peak_bytes"]
    low = smallest_feasible_budget(lib, g, peak)
    prev = 0
    for k in range(8, -1, -1):  # from the whole-graph peak down to the smallest feasible budget
        st = lib.harp_partition_plan(g.n, g.src, g.dst, low + (peak - low) * k // 8)[0]
        assert st["tri_blocks"] + st["wedge_blocks"] >= prev
        prev = st["tri_blocks"] + st["wedge_blocks"]
    assert prev > 2


def test_infeasible_budget_and_bad_arguments(lib):
    g = graphgen.ba(20_000, 4, 2)
    with pytest.raises(lib.HarpError) as ei:
        lib.harp_partition_plan(g.n, g.src, g.dst, 1 << 20)  # the per-vertex arrays alone exceed 1 MiB
    assert ei.value.status == lib.HARP_ENOMEM
    with pytest.raises(lib.HarpError) as ei:
        lib.harp_partition_plan(g.n, g.src, g.dst, 1 << 40, parts=-1)
    assert ei.value.status == lib.HARP_EINVAL
    with pytest.raises(lib.HarpError) as ei:
        lib.harp_partition_plan(3, np.array([0, 3], np.int32), np.array([1, 2], np.int32), 1 << 30)
    assert ei.value.status == lib.HARP_EINVAL
    import ctypes
    st = lib.harp_partition_stats()
    L = lib.lib()
    assert L.harp_partition_plan(5, 0, None, None, 1 << 30, 0, None, None, None, 0) == lib.HARP_EINVAL
    assert L.harp_partition_plan(5, 0, None, None, 1 << 30, 0, ctypes.byref(st), None, None, 4) == lib.HARP_EINVAL
    assert L.harp_partition_plan(5, 0, None, None, 1 << 30, 0, ctypes.byref(st), None, None, 0) == lib.HARP_OK
    assert (st.tri_blocks, st.wedge_blocks, st.m) == (1, 1, 0)


def test_edgeless_and_empty_graphs(lib):
    e = np.zeros(0, np.int32)
    for n in (0, 1, 6):
        st, tri, wedge = lib.harp_partition_plan(n, e, e, 1 << 30)
        assert st["m"] == 0
        if n:
            check_tiling(n, tri, wedge)


def test_zero_budget_needs_a_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present: a zero budget is sized from its free memory")
    g = graphgen.ba(100, 2, 1)
    with pytest.raises(lib.HarpError) as ei:
        lib.harp_partition_plan(g.n, g.src, g.dst, 0)
    assert ei.value.status == lib.HARP_ECUDA


def rank_graph_reference(n, src, dst):
    """Definition of the rank-order simple graph: drop self-loops and duplicates, rank = position of
    (degree, id) in lexicographic order, rows of the symmetric CSR sorted by rank."""
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    lo, hi = np.minimum(s, d)[keep], np.maximum(s, d)[keep]
    key = np.unique(lo * max(n, 1) + hi)
    a, b = key // max(n, 1), key % max(n, 1)
    deg = np.bincount(np.concatenate([a, b]), minlength=n)
    order = np.lexsort((np.arange(n), deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    ru, rv = rank[np.concatenate([a, b])], rank[np.concatenate([b, a])]
    srt = np.lexsort((rv, ru))
    off = np.concatenate([[0], np.cumsum(np.bincount(ru, minlength=n))])
    return rank, off, rv[srt]


def _messy_graph(n, m, seed):
    """Uniform random pairs with repeated edges (both orientations), self-loops and isolated vertices."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, m)
    d = rng.integers(0, n, m)
    rep = rng.integers(0, m, m // 4)
    s = np.concatenate([s, d[rep], s[: m // 10]])
    d = np.concatenate([d, s[rep], s[: m // 10]])  # reversed repeats and self-loops
    return s.astype(np.int32), d.astype(np.int32)


@pytest.mark.parametrize("case", ["messy_small", "messy_mid", "messy_dense", "hub_repeats", "ba", "chung_lu", "rmat",
                                  "empty", "edgeless"])
def test_host_rank_graph_is_the_definition(lib, case):
    if case == "messy_small":
        n, (s, d) = 50, _messy_graph(50, 300, 1)
    elif case == "messy_mid":
        n, (s, d) = 30_000, _messy_graph(30_000, 400_000, 2)
    elif case == "messy_dense":  # about 400 repeats per simple edge
        n, (s, d) = 300, _messy_graph(300, 2_000_000, 3)
    elif case == "hub_repeats":  # one row of 300,000 arcs with 1,000 distinct neighbours, both orientations
        x = (np.arange(300_000, dtype=np.int32) % 1000 + 1).astype(np.int32)
        n, s, d = 1001, np.concatenate([np.zeros_like(x), x]), np.concatenate([x, np.zeros_like(x)])
    elif case == "empty":
        n, s, d = 0, np.zeros(0, np.int32), np.zeros(0, np.int32)
    elif case == "edgeless":
        n, s, d = 17, np.zeros(0, np.int32), np.zeros(0, np.int32)
    else:
        g = {"ba": lambda: graphgen.ba(20_000, 6, 4), "chung_lu": lambda: graphgen.chung_lu(80_000, 2.1, 5000, 8, 9),
             "rmat": lambda: graphgen.rmat(15, 16, seed=3)}[case]()
        n, s, d = g.n, g.src, g.dst
    rank, off, cols = lib.harp_rank_csr_host(n, s, d)
    want_rank, want_off, want_cols = rank_graph_reference(n, s, d)
    assert np.array_equal(rank, want_rank)
    assert np.array_equal(off, want_off)
    assert np.array_equal(cols, want_cols)


def test_host_rank_graph_rejects_bad_ids(lib):
    with pytest.raises(lib.HarpError) as ei:
        lib.harp_rank_csr_host(4, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    assert ei.value.status == lib.HARP_EINVAL
    with pytest.raises(lib.HarpError) as ei:
        lib.harp_rank_csr_host(4, np.array([0, -1], np.int32), np.array([1, 2], np.int32))
    assert ei.value.status == lib.HARP_EINVAL
