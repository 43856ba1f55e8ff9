"""GPU parity: libharp (through its C ABI) against the CPU oracle, bit-exact uint64.

Inputs are seeded and synthetic (graphgen).  Sizes span every execution mode of every kernel:
warp-local and CTA triangle anchors, the fallback for out-degree > 1024, the three row-sort tiers,
and the warp / CTA-hash / windowed wedge modes; plus the full R-MAT scale-20 workload against
stored oracle counts.
"""
import json
import math
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import closed_forms, complete, edges_of, kbip  # noqa: E402

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


def gpu_count(H, n, src, dst, plan=None, device_input=True):
    if device_input:
        s = torch.from_numpy(np.ascontiguousarray(src, dtype=np.int32)).cuda()
        d = torch.from_numpy(np.ascontiguousarray(dst, dtype=np.int32)).cuda()
    else:
        s, d = src, dst
    g = H.harp_build_csr(n, s, d)
    try:
        counts, stats = H.harp_count4_stats(g, plan)
    finally:
        g.close()
    return counts, stats


CLOSED = closed_forms(scale=2)


@pytest.mark.parametrize("name,n,e,want", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(harp, name, n, e, want):
    s, d = e
    counts, _ = gpu_count(harp, n, s, d)
    assert counts.tolist() == [w % 2**64 for w in want]


def _random_graphs():
    out = []
    for i in range(36):
        n = [12, 40, 150, 600, 2500][i % 5]
        k = [2.5, 6, 14, 30][i % 4]
        gen = (graphgen.er, graphgen.rgg, graphgen.ba)[i % 3]
        out.append(gen(n, k, 9000 + i) if gen is not graphgen.ba else gen(n, 1 + i % 8, 9000 + i))
    return out


def test_random_graphs_against_esu_and_stats(harp):
    for g in _random_graphs():
        counts, stats = gpu_count(harp, g.n, g.src, g.dst)
        assert counts.tolist() == O.count4_esu(g.n, g.src, g.dst).tolist(), g.name
        assert stats.tolist() == O.noninduced(g.n, g.src, g.dst).tolist(), g.name


def test_plain_workload_ba2000(harp):
    """Plain single graph: Barabasi-Albert n=2000, m=4, seed 1 (~8k edges) against ESU."""
    g = graphgen.ba_2000()
    counts, stats = gpu_count(harp, g.n, g.src, g.dst)
    assert counts.tolist() == O.count4_esu(g.n, g.src, g.dst).tolist()
    assert int(stats[7]) == 7990


def test_batch_like_members(harp):
    """Members of the 4,096-graph batch workload (ER / BA / RGG, n up to 20,000) against the oracle."""
    for seed in (0, 1, 2, 3, 4, 5, 11, 97, 1234, 4095):
        g = graphgen.batch_graph(seed)
        counts, _ = gpu_count(harp, g.n, g.src, g.dst)
        assert counts.tolist() == O.count4_combo(g.n, g.src, g.dst).tolist(), g.name


def test_dense_graphs_all_modes(harp):
    """Dense ER graphs: CTA triangle mode, CTA-hash and windowed wedge modes, 16-bit counters."""
    for n, k, seed in ((800, 300, 1), (3000, 700, 2), (1500, 1200, 3)):
        g = graphgen.er(n, k, seed)
        counts, stats = gpu_count(harp, g.n, g.src, g.dst)
        assert stats.tolist() == O.noninduced(g.n, g.src, g.dst).tolist(), g.name
        assert counts.tolist() == O.count4_combo(g.n, g.src, g.dst).tolist(), g.name


def test_rmat_scale16_live_oracle(harp):
    g = graphgen.rmat(16, 16, seed=3)
    counts, stats = gpu_count(harp, g.n, g.src, g.dst)
    assert stats.tolist() == O.noninduced(g.n, g.src, g.dst).tolist()
    assert counts.tolist() == O.count4_combo(g.n, g.src, g.dst).tolist()


def test_rmat_scale20_full_workload(harp):
    """The bench workload at full size against counts stored by tests/golden/make_golden_large.py."""
    with open(os.path.join(HERE, "golden", "rmat20_oracle.json")) as f:
        gold = json.load(f)
    g = graphgen.rmat_scale20()
    assert g.m_in == gold["m_in"]
    counts, stats = gpu_count(harp, g.n, g.src, g.dst)
    assert stats.tolist() == gold["stats"]
    assert counts.tolist() == gold["counts"]


def test_rmat_scale20_repeated_counts(harp):
    """Eight counts of the bench workload, each on a fresh handle (fresh workspace memory; device and
    host inputs alternating), all equal to the stored counts: a race or an undefined read in a kernel
    shows up as an occasional count that differs from the rest, which one count alone would catch
    only by chance."""
    with open(os.path.join(HERE, "golden", "rmat20_oracle.json")) as f:
        gold = json.load(f)
    g = graphgen.rmat_scale20()
    for k in range(8):
        counts, stats = gpu_count(harp, g.n, g.src, g.dst, device_input=(k % 2 == 0))
        assert stats.tolist() == gold["stats"], k
        assert counts.tolist() == gold["counts"], k


def test_host_and_device_inputs_agree(harp):
    g = graphgen.ba(3000, 6, 5)
    a, _ = gpu_count(harp, g.n, g.src, g.dst, device_input=True)
    b, _ = gpu_count(harp, g.n, g.src, g.dst, device_input=False)
    assert a.tolist() == b.tolist()


def test_invariances(harp):
    rng = np.random.default_rng(1)
    g = graphgen.ba(4000, 5, 77)
    want, _ = gpu_count(harp, g.n, g.src, g.dst)
    perm = rng.permutation(g.n).astype(np.int32)
    got, _ = gpu_count(harp, g.n, perm[g.src], perm[g.dst])
    assert got.tolist() == want.tolist()
    s = np.concatenate([g.src, g.dst, g.src[:50], np.arange(20, dtype=np.int32)])
    d = np.concatenate([g.dst, g.src, g.dst[:50], np.arange(20, dtype=np.int32)])
    o = rng.permutation(len(s))
    got, _ = gpu_count(harp, g.n, s[o], d[o])
    assert got.tolist() == want.tolist()
    got, _ = gpu_count(harp, g.n + 1000, g.src, g.dst)
    assert got.tolist() == want.tolist()


def test_plans_never_change_counts(harp):
    g = graphgen.rmat(14, 16, seed=9)
    want = O.count4_combo(g.n, g.src, g.dst).tolist()
    s = torch.from_numpy(g.src).cuda()
    d = torch.from_numpy(g.dst).cuda()
    csr = harp.harp_build_csr(g.n, s, d)
    try:
        chosen = harp.harp_select_anchors(csr)
        assert harp.harp_count4(csr, chosen).tolist() == want
        for wm, cm in ((32, 64), (64, 64), (512, 8192), (2, 2), (256, 600)):
            p = harp.harp_plan()
            p.version = harp.HARP_ABI_VERSION
            p.c4_warp_max_work = wm
            p.c4_cta_max_work = cm
            assert harp.harp_count4(csr, p).tolist() == want, (wm, cm)
        # the same handle counted again gives the same result
        assert harp.harp_count4(csr).tolist() == want
    finally:
        csr.close()


def test_empty_and_degenerate(harp):
    e = np.zeros(0, np.int32)
    for n in (0, 1, 5):
        counts, stats = gpu_count(harp, n, e, e, device_input=False)
        assert counts.tolist() == [0] * 6
    s, d = edges_of([(0, 1)])
    assert gpu_count(harp, 2, s, d)[0].tolist() == [0] * 6
    s, d = complete(3)
    assert gpu_count(harp, 3, s, d)[0].tolist() == [0] * 6
    s = np.array([0, 1, 1], np.int32)
    d = np.array([0, 1, 1], np.int32)  # only self-loops
    assert gpu_count(harp, 2, s, d)[0].tolist() == [0] * 6


def test_invalid_ids_raise(harp):
    with pytest.raises(harp.HarpError) as ei:
        gpu_count(harp, 3, np.array([0, 3], np.int32), np.array([1, 2], np.int32))
    assert ei.value.status == harp.HARP_EINVAL
    with pytest.raises(harp.HarpError):
        gpu_count(harp, 3, np.array([-1], np.int32), np.array([1], np.int32), device_input=False)


def test_async_entry_point_and_launch_count(harp):
    g = graphgen.ba(1000, 3, 4)
    s = torch.from_numpy(g.src).cuda()
    d = torch.from_numpy(g.dst).cuda()
    csr = harp.harp_build_csr(g.n, s, d)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    before = harp.harp_launch_count()
    harp.harp_count4_async(csr, out.data_ptr())
    torch.cuda.synchronize()
    assert harp.harp_launch_count() > before
    got = out.cpu().numpy().view(np.uint64)[:6]
    csr.close()
    assert got.tolist() == O.count4_esu(g.n, g.src, g.dst).tolist()


def test_large_grid_boundary_table(harp):
    """A grid of more than 15 windows per row keeps every 2^s-th boundary and finds the rest by a
    galloping search: 2e6 vertices of degree >= 2 span about 30 windows of 48 KiB (about 15 of 100 KiB,
    8 of 200 KiB); every window size (100 KiB for two 512-thread blocks per SM, the default; 200 KiB
    for one 1024-thread block; 64 and 48 KiB for 3 and 4 blocks of 512) agrees with the oracle."""
    g = graphgen.chung_lu(2_000_000, 2.1, 3000, 4, 5)
    want = O.count4_combo(g.n, g.src, g.dst).tolist()
    for bytes_ in (0, 204800, 65536, 49152):
        p = harp.harp_plan()
        p.version = harp.HARP_ABI_VERSION
        p.c4_window_bytes = bytes_
        assert harp.count4_edges(g.n, g.src, g.dst, p).tolist() == want, bytes_


def test_counter_widths_at_their_limits(harp):
    """Wedge counters are 3, 4, 5, 6, 8, 16 or 32 bits wide by the degree of x (cnt(x) <= d(x)).  In
    K_{k,k} (ranks = ids, all degrees k) the top root u has every vertex of the other side as a lower
    neighbour, so every x on u's side below u reaches cnt(x) = d(x) = k: k = 2^b - 1 fills a b-bit
    counter exactly and k = 2^b moves x into the next band.  K_{2,k} does the same for the 16-bit
    band's limit and the 32-bit band.  c4_warp_max_work = 1 sends every root with wedge work to the
    windowed counters; with and without band merging the counts are the closed forms."""
    cases = [(k, k) for k in (7, 8, 15, 16, 31, 32, 63, 64, 255, 256)] + [(2, 65535), (2, 65536)]
    for a, b in cases:
        s, d = kbip(a, b)
        want = [a * math.comb(b, 3) + b * math.comb(a, 3), 0, 0, math.comb(a, 2) * math.comb(b, 2), 0, 0]
        for flags in (0, harp.HARP_PLAN_NO_BAND_MERGE):
            p = harp.harp_plan()
            p.version = harp.HARP_ABI_VERSION
            p.c4_warp_max_work = 1
            p.flags = flags
            got, _ = gpu_count(harp, a + b, s, d, plan=p)
            assert got.tolist() == want, (a, b, flags)


def test_band_merging_never_changes_counts(harp):
    """A heavy-tailed graph whose x-range has every counter band: merged or separate bands, and the
    windowed or the warp-hash mode for small roots, all give the oracle's counts."""
    g = graphgen.chung_lu(100_000, 2.1, 2000, 6, 11)
    want = O.count4_combo(g.n, g.src, g.dst).tolist()
    for wm in (0, 1):
        for flags in (0, harp.HARP_PLAN_NO_BAND_MERGE):
            p = harp.harp_plan()
            p.version = harp.HARP_ABI_VERSION
            p.c4_warp_max_work = wm
            p.flags = flags
            assert harp.count4_edges(g.n, g.src, g.dst, p).tolist() == want, (wm, flags)


def test_wedge_middle_tier_never_changes_counts(harp):
    """Roots with wedge work between the warp limit and c4_cta_max_work (at most 2048) take the middle
    tier (a 4096-slot warp hash) instead of the windows: off, default, and every root up to 2048 wedges
    in it (warp limit 1) all give the oracle's counts, on a skewed and a flat graph."""
    for g in (graphgen.rmat(15, 16, seed=21), graphgen.chung_lu(60000, 2.1, 2500, 10, 8), graphgen.er(20000, 24, 3)):
        want = O.count4_combo(g.n, g.src, g.dst).tolist()
        for wm, mid in ((0, 1), (0, 0), (1, 2048), (256, 1024)):
            p = harp.harp_plan()
            p.version = harp.HARP_ABI_VERSION
            p.c4_warp_max_work = wm
            p.c4_cta_max_work = mid
            assert harp.count4_edges(g.n, g.src, g.dst, p).tolist() == want, (g.name, wm, mid)
