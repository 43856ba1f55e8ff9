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
