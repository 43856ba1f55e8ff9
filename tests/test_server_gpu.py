"""Continuous-batching server (GPU): every request gets exactly the counts it gets alone, whatever it
was batched with, from one thread or several, under a budget small enough to make requests queue, and
a request larger than the budget is counted by the partitioned path."""
import threading

import numpy as np
import pytest

import graphgen

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


def mix(count, seed0):
    gs = []
    for i in range(count):
        gs.append(graphgen.batch_graph(seed0 + i, n_lo=50, n_hi=6000))
    gs.append(graphgen.rmat(13, 16, seed=seed0))
    return gs


def test_results_equal_alone_and_in_the_mix(harp):
    gs = mix(60, 100)
    alone = [harp.count4_edges(g.n, g.src, g.dst) for g in gs]
    srv = harp.Server(hbm_budget_bytes=1 << 30, batch_window_us=500_000)
    try:
        tickets = [srv.submit(g.n, g.src, g.dst) for g in gs]
        for t, want in zip(tickets, alone):
            assert srv.wait(t).tolist() == want.tolist()
        st = srv.stats()
        assert st["completed"] == len(gs)
        assert st["batches"] < len(gs)           # requests were batched together
        assert st["max_batch"] > 1
        assert 0 < st["latency_p50_us"] <= st["latency_p99_us"]
        with pytest.raises(harp.HarpError) as ei:
            srv.poll(tickets[0])                 # retired
        assert ei.value.status == harp.HARP_ENOTFOUND
    finally:
        srv.close()


def test_concurrent_submitters_and_small_budget(harp):
    gs = mix(40, 300)
    alone = {k: harp.count4_edges(g.n, g.src, g.dst) for k, g in enumerate(gs)}
    biggest = max(g.m_in for g in gs)
    budget = 96 * biggest + (4 << 20)            # the largest request fits; the mix has to queue
    srv = harp.Server(hbm_budget_bytes=budget, max_inflight=8, batch_window_us=2000)
    results, errors = {}, []

    def worker(ids):
        try:
            tickets = [(k, srv.submit(gs[k].n, gs[k].src, gs[k].dst)) for k in ids]
            for k, t in tickets:
                while True:
                    r = srv.poll(t)
                    if r is not None:
                        results[k] = r
                        break
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(list(range(j, len(gs), 4)),)) for j in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    srv_stats = srv.stats()
    srv.close()
    assert not errors, errors
    assert {k: v.tolist() for k, v in results.items()} == {k: v.tolist() for k, v in alone.items()}
    assert srv_stats["peak_resident_bytes"] <= budget
    assert srv_stats["partitioned"] == 0


def test_oversize_request_uses_partitions_and_bad_request_fails(harp):
    g = graphgen.rmat(14, 16, seed=8)
    want = harp.count4_edges(g.n, g.src, g.dst)
    srv = harp.Server(hbm_budget_bytes=12 << 20)   # below this request's footprint
    try:
        t = srv.submit(g.n, g.src, g.dst)
        assert srv.wait(t).tolist() == want.tolist()
        assert srv.stats()["partitioned"] == 1
        bad = srv.submit(3, np.array([0, 7], np.int32), np.array([1, 2], np.int32))
        with pytest.raises(harp.HarpError) as ei:
            srv.wait(bad)
        assert ei.value.status == harp.HARP_EINVAL
        with pytest.raises(harp.HarpError):
            srv.poll(123456789)
    finally:
        srv.close()


def test_small_requests_do_not_wait_behind_a_large_one(harp):
    """Small requests take the second, higher-priority lane: submitted right after a large request
    (R-MAT scale 20, about 16M input pairs), most of them finish before it, and every result is the
    request's alone-count.  With a single lane (small_edges = 0xFFFFFFFF) the counts are the same."""
    big = graphgen.rmat(20, 16, seed=31)
    smalls = [graphgen.batch_graph(900 + i, n_lo=50, n_hi=3000) for i in range(24)]
    want_big = harp.count4_edges(big.n, big.src, big.dst).tolist()
    want_small = [harp.count4_edges(g.n, g.src, g.dst).tolist() for g in smalls]
    assert all(g.m_in <= 65536 for g in smalls) and big.m_in > 65536
    for small_edges in (0, 0xFFFFFFFF):
        srv = harp.Server(small_edges=small_edges)
        try:
            tb = srv.submit(big.n, big.src, big.dst)
            ts = [srv.submit(g.n, g.src, g.dst) for g in smalls]
            done, order = {}, []
            while len(done) < len(ts) + 1:
                for t in [tb] + ts:
                    if t in done:
                        continue
                    r = srv.poll(t)
                    if r is not None:
                        done[t] = r.tolist()
                        order.append(t)
            assert done[tb] == want_big
            assert [done[t] for t in ts] == want_small
            if small_edges == 0:
                before = sum(1 for t in order[:order.index(tb)] if t in ts)
                assert before >= 0.75 * len(ts), (before, len(ts))
        finally:
            srv.close()
