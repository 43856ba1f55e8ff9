"""Batched counting on the GPU: every member of a batch must get exactly its own counts (the batch is
the disjoint union of its members, so an occurrence never spans two of them), whether the batch is
counted through its captured CUDA graph, replayed, re-captured for another plan, or launched
kernel by kernel."""
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


def members():
    out = []
    for seed in range(40):
        g = graphgen.batch_graph(seed)
        out.append((g.n, g.src, g.dst, g.name))
    for name, (n, e) in {"K40": (40, complete(40)), "K1100": (1100, complete(1100)), "W5000": (5001, wheel(5000)),
                         "K300,500": (800, kbip(300, 500)), "CP40": (80, cocktail(40))}.items():
        out.append((n, e[0], e[1], name))
    z = np.zeros(0, np.int32)
    out.append((0, z, z, "empty"))
    out.append((7, z, z, "edgeless"))
    out.append((2, np.array([0], np.int32), np.array([1], np.int32), "one edge"))
    return out


@pytest.fixture(scope="module")
def handles(harp):
    hs, alone, info = [], [], []
    for n, s, d, name in members():
        h = harp.harp_build_csr(n, s, d)
        hs.append(h)
        c, st = harp.harp_count4_stats(h)
        alone.append(c)
        info.append((n, s, d, name, st))
    yield hs, np.array(alone), info
    for h in hs:
        h.close()


def test_batch_equals_members_alone(harp, handles):
    hs, alone, info = handles
    b = harp.harp_batch_create(hs)
    try:
        counts, stats = harp.harp_batch_count(b, stats=True)
        assert counts.tolist() == alone.tolist()
        for k, (_, _, _, name, st) in enumerate(info):
            assert stats[k].tolist() == st.tolist(), name
        again = harp.harp_batch_count(b)              # replay of the captured graph
        assert again.tolist() == alone.tolist()
        p = harp.harp_plan()
        p.version = harp.HARP_ABI_VERSION
        p.flags = harp.HARP_PLAN_NO_GRAPH
        assert harp.harp_batch_count(b, p).tolist() == alone.tolist()
        p2 = harp.harp_plan()
        p2.version = harp.HARP_ABI_VERSION
        p2.c4_warp_max_work = 16
        p2.c4_cta_max_work = 64
        assert harp.harp_batch_count(b, p2).tolist() == alone.tolist()  # re-captured for a new plan
        inf = harp.harp_batch_info(b)
        assert inf["graphs"] == len(hs)
    finally:
        b.close()


def test_batch_members_against_oracle(harp, handles):
    hs, alone, info = handles
    for k, (n, s, d, name, _) in enumerate(info):
        if n <= 6000:
            assert alone[k].tolist() == O.count4_combo(n, s, d).tolist(), name


def test_one_shot_batch_and_member_order(harp, handles):
    hs, alone, _ = handles
    order = list(range(len(hs)))[::-1]
    got = harp.harp_count4_batch([hs[i] for i in order])
    assert got.tolist() == alone[order].tolist()
    assert harp.harp_count4_batch([]).shape == (0, 6)


def test_autotune_grid_and_custom_candidates(harp, handles):
    hs, alone, _ = handles
    b = harp.harp_batch_create(hs)
    try:
        base = harp.harp_batch_count(b)
        assert base.tolist() == alone.tolist()
        best, ms = harp.harp_batch_autotune(b, reps=1)
        timed = [x for x in ms if x > 0]
        # the per-degree-bin descent: the default plan, then 2 + 4 x 2 + 3 + 2 + 2 knob values, each
        # distinct plan timed once (at least one value of every knob equals the current plan)
        assert len(ms) == harp.HARP_AUTOTUNE_GRID and 7 <= len(timed) <= 18
        assert ms[len(timed):] == [0.0] * (len(ms) - len(timed))
        assert best.tri_warp_max in (16, 32) and best.c4_warp_max_work in (256, 512)
        assert best.tri_cta_max in (256, 512, 1024) and best.c4_window_bytes in (0, 100 * 1024, 200 * 1024)
        assert all(v in (harp.HARP_PROBE_HASH, harp.HARP_PROBE_BSEARCH) for v in best.tri_probe_bin)
        assert harp.harp_batch_count(b, best).tolist() == base.tolist()
        cands = []
        for wm, cta in ((4, 64), (32, 1024)):
            p = harp.harp_plan()
            p.version = harp.HARP_ABI_VERSION
            p.tri_warp_max, p.tri_cta_max = wm, cta
            cands.append(p)
        best2, ms2 = harp.harp_batch_autotune(b, cands, reps=2)
        assert len(ms2) == 2 and all(x > 0 for x in ms2)
        assert (best2.tri_warp_max, best2.tri_cta_max) in ((4, 64), (32, 1024))
        assert harp.harp_batch_count(b, best2).tolist() == base.tolist()
    finally:
        b.close()


def test_every_per_bin_variant_counts_the_same(harp, handles):
    """Each knob of the per-degree-bin search on its own (the probe of every triangle bin, the warp/CTA
    splits, the staging capacity, the wedge window) gives the alone-counts of every member, batched and
    one graph at a time."""
    hs, alone, _ = handles
    b = harp.harp_batch_create(hs)
    try:
        variants = []
        for binno in range(4):
            for probe in (harp.HARP_PROBE_HASH, harp.HARP_PROBE_BSEARCH):
                p = harp.harp_plan()
                p.version = harp.HARP_ABI_VERSION
                p.tri_probe_bin[binno] = probe
                p.tri_probe = harp.HARP_PROBE_BSEARCH if probe == harp.HARP_PROBE_HASH else harp.HARP_PROBE_HASH
                variants.append(p)
        for field, values in (("tri_warp_max", (8, 16)), ("tri_cta_max", (256, 512)),
                              ("c4_warp_max_work", (64, 256)), ("c4_window_bytes", (200 * 1024, 64 * 1024))):
            for v in values:
                p = harp.harp_plan()
                p.version = harp.HARP_ABI_VERSION
                setattr(p, field, v)
                variants.append(p)
        for p in variants:
            assert harp.harp_batch_count(b, p).tolist() == alone.tolist(), p.as_dict()
        for k in (0, len(hs) // 2, len(hs) - 1):
            assert harp.harp_count4(hs[k], variants[3]).tolist() == alone[k].tolist()
    finally:
        b.close()
