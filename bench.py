"""Benchmark: exact induced 4-motif counts, edges/s on one GB300 (and N replicas under torchrun).

Workload (default): the plain single large skewed graph, R-MAT scale 20, edge factor 16,
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05), seed 1, symmetrised with self-loops and duplicates removed
(m = 15,702,112 undirected edges).  One step = one harp_count4 on the device-resident CSR: degree
ordering + relabelled CSR, triangle / 4-clique anchors with per-edge t_e, wedge anchors (4-cycles),
reduction and closure, counts copied to the host.  L2 is flushed (256 MiB write) between steps.

`value` = m / (device time per step).  `e2e` = the same metric through the public API from pinned
host edge lists: harp_build_csr (H2D + device CSR build) + harp_count4 (D2H of the counts) per step.
`roofline` = the dominant kernel's algorithmic bytes (host work meter) / its CUDA-event time, against
the measured HBM copy bandwidth (`segment_rooflines`: the same for every segment).  `cpu_baseline` =
the CPU oracle (OpenMP, all host cores) on the bench graph itself.

`batched`: the batched workload (4,096 graphs: ER / BA / RGG, n log-uniform in [50, 20000], mean degree
in [4, 32], seeds 0..4095) counted as one captured CUDA graph under the autotuned plan, against the plain
path (one harp_count4 per graph) over the same graphs; counts are compared graph by graph.
`served`: a Poisson stream of requests (edge counts log-uniform in [1e3, 1e7], ER / BA / RGG / R-MAT)
through the continuous-batching server, against plain one-graph-per-launch processing (build + count,
in arrival order) of the same stream: p50 / p99 latency and edges/s.

`partitioned`: the partitioned large graph (Chung-Lu, exponent 2.1, max expected degree 1e6, mean degree
48; n = 5e7 gives about 1.2e9 edges) counted once through harp_count4_partitioned under a 24 GiB device
cap, with edges/s over the whole call (host edge list to counts) and its host / transfer / kernel split,
and the same graph counted whole on the device without a cap: `partitioned_equals_whole` is the owner
rule's exactness check at full size.  `--workload partitioned` prints it as its own line; `--n`
shrinks the graph for trial runs.

--impl reference runs the CPU oracle (plain non-induced counts + containment inversion) on the host
cores instead: each step counts an R-MAT scale-17 sample of the same family.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges/s, exact induced 4-motif counts (batched vs plain, 1 GB300); % HBM peak"
UNIT = "edges/s"
SEGMENTS = ("orient", "tri_warp", "tri_cta_small", "tri_cta_large", "tri_fallback", "c4_small", "c4_mid",
            "c4_window", "reduce")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples: kept in HARP_CLOCKS_DIR when it is set, else a temporary file (the JSON line
        # carries the summary)
        keep = os.environ.get("HARP_CLOCKS_DIR")
        self.keep = bool(keep)
        self.path = None
        if keep:
            self.path = os.path.join(keep, f"clocks_bench_{os.getpid()}.csv")
        elif shutil.which("nvidia-smi"):
            fd, self.path = tempfile.mkstemp(prefix="harp_clocks_", suffix=".csv")
            os.close(fd)

    def __enter__(self):
        if self.path is None:
            return self
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            if not self.keep and self.path and os.path.exists(self.path):
                os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not self.keep:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu on Arm, /proc/cpuinfo on x86), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample_rate(scale: int, threads: int = 0, counts: bool = False):
    """Time the CPU oracle on an R-MAT graph of the bench family in a fresh process (OpenMP on all
    host cores).  counts=True also returns the oracle's counts (as a check against the GPU's)."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import graphgen, oracle, os\n"
        "g = graphgen.rmat(%d, 16, 0.57, 0.19, 0.19, seed=1)\n"
        "m, _ = oracle.graph_summary(g.n, g.src, g.dst)\n"
        "t = time.perf_counter(); c = oracle.count4_combo(g.n, g.src, g.dst, %d); t = time.perf_counter() - t\n"
        "print(json.dumps({'m': m, 'seconds': t, 'cores': os.cpu_count(), 'counts': [int(x) for x in c]}))\n"
        % (ROOT, scale, threads))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    if not counts:
        r.pop("counts", None)
    return r


def oracle_a_rate():
    """Oracle A (Wernicke's ESU over every connected 4-subset, one thread) on the plain small graph
    (Barabasi-Albert n = 2000, 4 edges per new vertex, seed 1), in a fresh process."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import graphgen, oracle\n"
        "g = graphgen.ba_2000()\n"
        "m, _ = oracle.graph_summary(g.n, g.src, g.dst)\n"
        "t = time.perf_counter(); c = oracle.count4_esu(g.n, g.src, g.dst, 1); t = time.perf_counter() - t\n"
        "print(json.dumps({'m': m, 'seconds': t, 'counts': [int(x) for x in c]}))\n" % (ROOT,))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def max_over_ranks(value: float, world: int, device: str) -> float:
    """The largest value over all ranks (a replicated job takes as long as its slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(m: int, world: int, step_ms: float) -> float:
    """Whole-job edges/s of `world` replicas that each count the m-edge graph in step_ms (the max)."""
    return world * m / (step_ms / 1000.0)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    scale = 17
    times, m = [], None
    for _ in range(args.warmup):
        oracle_sample_rate(scale)
    for _ in range(args.steps):
        r = oracle_sample_rate(scale)
        times.append(r["seconds"])
        m = r["m"]
        cores = r["cores"]
    t = sum(times) / len(times)
    value = m / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "rmat(scale=17, ef=16, a=0.57, b=0.19, c=0.19, seed=1) sample of the "
                                   "R-MAT scale-20 family", "graph_edges": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"R-MAT scale 17 (m={m}) per step, oracle count4_combo"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batched(harp, graphgen, np, torch, stream, flush, steps, warmup, G=4096):
    """Batched vs plain on the 4,096-graph workload (both exact; counts compared per graph)."""
    t0 = time.perf_counter()
    gs = [graphgen.batch_graph(s) for s in range(G)]
    t_gen = time.perf_counter() - t0
    csrs = [harp.harp_build_csr(g.n, g.src, g.dst) for g in gs]
    m_total = sum(c.info()["m"] for c in csrs)
    b = harp.harp_batch_create(csrs)
    best, tune_ms = harp.harp_batch_autotune(b, reps=2)
    for _ in range(warmup):
        counts_b = harp.harp_batch_count(b, best, stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        counts_b = harp.harp_batch_count(b, best, stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_b = sum(a.elapsed_time(z) for a, z in ev) / steps
    # plain: one graph per launch sequence, same graphs and plan, one untimed pass then one timed pass
    for c in csrs:
        harp.harp_count4(c, best)
    flush.fill_(1)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plain = [harp.harp_count4(c, best) for c in csrs]
    z.record(stream)
    torch.cuda.synchronize()
    t_p = a.elapsed_time(z)
    assert all(np.array_equal(p, q) for p, q in zip(plain, counts_b)), "batched counts differ from plain"
    info = harp.harp_batch_info(b)
    b.close()
    for c in csrs:
        c.close()
    return {"workload": f"{G} graphs, ER/BA/RGG uniform, n log-uniform [50, 20000], mean degree U[4, 32] "
                        f"(BA m in 2..8), seeds 0..{G - 1}", "graphs": G, "n_total": info["n"], "m_total": m_total,
            "value": m_total / (t_b / 1000), "unit": UNIT, "ms_per_step": t_b,
            "plain_value": m_total / (t_p / 1000), "plain_ms_per_pass": t_p, "speedup_vs_plain": t_p / t_b,
            "plan": {"tri_warp_max": best.tri_warp_max,
                     "tri_probe_bin": {name: ("bsearch" if v == harp.HARP_PROBE_BSEARCH else "hash")
                                       for name, v in zip(("warp", "cta256", "cta512", "cta1024"),
                                                          list(best.tri_probe_bin))},
                     "tri_cta_max": best.tri_cta_max, "c4_warp_max_work": best.c4_warp_max_work,
                     "c4_window_bytes": best.c4_window_bytes},
            "autotune_ms": [t for t in tune_ms if t > 0], "generate_s": t_gen, "counts_equal": True}


def bench_served(harp, graphgen, np, rates=(10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0), nreq=1000, seed=11,
                 budget=64 << 30):
    """Poisson streams (one per rate, the same requests) through the server vs plain processing."""
    t0 = time.perf_counter()
    gs = [graphgen.serve_graph(seed * 100000 + i) for i in range(nreq)]
    t_gen = time.perf_counter() - t0
    # warm-up: build and count one request of each generator family once, untimed
    for g in {g.name.split("(")[0]: g for g in gs[:64]}.values():
        c = harp.harp_build_csr(g.n, g.src, g.dst)
        harp.harp_count4(c)
        c.close()
    out = {"workload": f"{nreq} requests per rate, Poisson arrivals, edge counts log-uniform [1e3, 1e7], "
                       f"ER/BA/RGG/R-MAT uniform, HBM budget {budget >> 30} GiB", "requests": nreq,
           "lanes": "small requests (<= 65536 input pairs) on a second, higher-priority compute stream",
           "generate_s": t_gen, "rates": []}
    for k, rate in enumerate(rates):
        r = served_at_rate(harp, np, gs, rate, seed + k, budget)
        out["rates"].append(r)
        out["edges"] = r.pop("edges")
    top = out["rates"][-1]  # the saturated stream: throughput of the path, not of the arrivals
    out.update({"value": top["value"], "unit": UNIT, "plain_value": top["plain_value"], "at_rate": top["rate"],
                "counts_equal": True})
    return out


def served_at_rate(harp, np, gs, rate, seed, budget):
    import threading
    nreq = len(gs)
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    alone = [None] * nreq
    m_of = [0] * nreq

    def plain_pass():
        lat = []
        t0 = time.perf_counter()
        for i, g in enumerate(gs):
            now = time.perf_counter() - t0
            if now < arrivals[i]:
                time.sleep(arrivals[i] - now)
            c = harp.harp_build_csr(g.n, g.src, g.dst)
            alone[i] = harp.harp_count4(c)
            m_of[i] = c.info()["m"]
            c.close()
            lat.append(time.perf_counter() - t0 - arrivals[i])
        return lat, time.perf_counter() - t0

    lat_p, span_p = plain_pass()
    srv = harp.Server(hbm_budget_bytes=budget)
    tickets = [None] * nreq
    done_at = [0.0] * nreq
    t0 = time.perf_counter()

    def submitter():
        for i, g in enumerate(gs):
            now = time.perf_counter() - t0
            if now < arrivals[i]:
                time.sleep(arrivals[i] - now)
            tickets[i] = srv.submit(g.n, g.src, g.dst)

    th = threading.Thread(target=submitter)
    th.start()
    results = [None] * nreq
    pending = set(range(nreq))
    while pending:
        for i in list(pending):
            if tickets[i] is None:
                continue
            r = srv.poll(tickets[i])
            if r is not None:
                results[i] = r
                done_at[i] = time.perf_counter() - t0
                pending.discard(i)
        time.sleep(0.0002)
    th.join()
    span_s = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    assert all(np.array_equal(r, a) for r, a in zip(results, alone)), "served counts differ from plain"
    lat_s = [done_at[i] - arrivals[i] for i in range(nreq)]
    m_total = sum(m_of)
    pct = lambda v, q: float(np.percentile(np.asarray(v) * 1000.0, q))
    return {"rate": rate, "edges": m_total, "value": m_total / span_s,
            "p50_ms": pct(lat_s, 50), "p99_ms": pct(lat_s, 99),
            "plain_value": m_total / span_p, "plain_p50_ms": pct(lat_p, 50), "plain_p99_ms": pct(lat_p, 99),
            "batches": st["batches"], "max_batch": st["max_batch"], "partitioned": st["partitioned"],
            "peak_resident_bytes": st["peak_resident_bytes"]}


def bench_partitioned(harp, graphgen, torch, n, cap_gib, steps=1, warmup=0, whole=True):
    """The partitioned large-graph workload (Chung-Lu, exponent 2.1, max expected degree 1e6, mean
    degree 48; n = 5e7 gives about 1.2e9 edges): harp_count4_partitioned under a device cap, timed
    from the host edge list to the counts (Table IV's split: host / transfer / kernels), and the same
    graph counted whole on the device (harp_build_csr from device-resident edges + harp_count4, no
    cap) as the exactness check of the owner rule: the two counts must be equal."""
    t0 = time.perf_counter()
    g = graphgen.chung_lu_large(n)
    t_gen = time.perf_counter() - t0
    budget = int(cap_gib * (1 << 30))
    runs = []
    for k in range(warmup + steps):
        t = time.perf_counter()
        counts, st = harp.harp_count4_partitioned(g.n, g.src, g.dst, budget_bytes=budget)
        wall = time.perf_counter() - t
        if k >= warmup:
            runs.append((wall, st, counts))
    wall, st, counts = min(runs, key=lambda r: r[0])
    m = st["m"]
    out = {"workload": f"chung_lu(n={g.n}, gamma=2.1, max expected degree {1e6 * g.n / 5e7:g}, mean degree 48, "
                       f"seed 1), partitioned under a {cap_gib:g} GiB device cap",
           "n": g.n, "m": m, "value": m / wall, "unit": UNIT, "seconds": wall, "runs": len(runs),
           "blocks": st["partitions"], "tri_blocks": st["tri_blocks"], "wedge_blocks": st["wedge_blocks"],
           "wedge_sliced": st["wedge_sliced"], "device_peak_bytes": st["device_peak_bytes"],
           "halo_arcs": st["halo_arcs"], "h2d_bytes": st["h2d_bytes"], "host_ms": st["host_ms"],
           "host_graph_ms": st["graph_ms"], "host_cut_ms": st["cut_ms"], "device_tri_ms": st["tri_ms"],
           "device_wedge_ms": st["wedge_ms"], "transfer_ms": st["transfer_ms"], "device_ms": st["device_ms"],
           "transfer_share": st["transfer_ms"] / (1000 * wall), "generate_s": t_gen,
           "counts": [int(x) for x in counts]}
    if whole:
        # the same edges whole on the device: no cap, one CSR, one count (per-segment CUDA events)
        t = time.perf_counter()
        src_d = torch.from_numpy(g.src).cuda()
        dst_d = torch.from_numpy(g.dst).cuda()
        csr = harp.harp_build_csr(g.n, src_d, dst_d)
        del src_d, dst_d
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t
        harp.harp_set_profiling(True)
        t = time.perf_counter()
        cw = harp.harp_count4(csr)
        t_count = time.perf_counter() - t
        ms, _ = harp.harp_last_stage_times()
        harp.harp_set_profiling(False)
        info = csr.info()
        csr.close()
        torch.cuda.empty_cache()
        out["whole"] = {"m": info["m"], "device_bytes": info["device_bytes"], "build_s": t_build,
                        "count_s": t_count, "value": info["m"] / t_count, "unit": UNIT,
                        "segments_ms": {k: v for k, v in zip(SEGMENTS, ms)}, "counts": [int(x) for x in cw]}
        out["partitioned_equals_whole"] = [int(x) for x in cw] == out["counts"] and info["m"] == m
    return out


def run_partitioned(args):
    """The partitioned large-graph workload as its own JSON line (edges/s of the partitioned call)."""
    import torch

    import graphgen
    from paper_2607_12074_gb300 import _build, harp

    world, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    _build.build()
    harp.lib()
    with ClockSampler(local) as clocks:
        r = bench_partitioned(harp, graphgen, torch, args.n, args.cap_gib, steps=args.steps, warmup=args.warmup,
                              whole=not args.no_whole)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["runs"],
            "warmup": args.warmup, "ms_per_step": 1000 * r["seconds"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": r["workload"], "n": r["n"], "m": r["m"], "parallelism": "single",
                       "l2": "inputs larger than L2"},
            "partitioned": r, "clocks": clocks.summary(), "counts": r["counts"]}
    print(json.dumps(line), flush=True)
    return 0


def run_whole(args):
    """The same heavy-tailed family as the partitioned workload, counted whole on the device: the CSR is
    built from device-resident edges, then each step is one harp_count4 with per-segment CUDA-event
    times (the CSR, well above L2, is read from HBM every step)."""
    import torch

    import graphgen
    from paper_2607_12074_gb300 import _build, harp

    world, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    _build.build()
    harp.lib()
    t0 = time.perf_counter()
    g = graphgen.chung_lu_large(args.n)
    t_gen = time.perf_counter() - t0
    csr = harp.harp_build_csr(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
    m = csr.info()["m"]
    harp.harp_set_profiling(True)
    plan = None
    if args.c4_window_kib:
        plan = harp.harp_plan()
        plan.version = harp.HARP_ABI_VERSION
        plan.c4_window_bytes = int(args.c4_window_kib * 1024)
    runs = []
    for k in range(args.warmup + args.steps):
        with ClockSampler(local) as clocks:
            counts = harp.harp_count4(csr, plan)
            ms, _ = harp.harp_last_stage_times()
        if k >= args.warmup:
            runs.append((sum(ms), ms, clocks.summary()))
    harp.harp_set_profiling(False)
    csr.close()
    total, ms, clk = min(runs, key=lambda r: r[0])
    line = {"metric": METRIC, "value": m / (total / 1000), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"chung_lu(n={g.n}, gamma=2.1, max expected degree {1e6 * g.n / 5e7:g}, "
                                   f"mean degree 48, seed 1), whole graph on the device",
                       "n": g.n, "m": m, "parallelism": "single", "l2": "inputs larger than L2"},
            "segments_ms": {k: v for k, v in zip(SEGMENTS, ms)}, "generate_s": t_gen, "clocks": clk,
            "c4_window_kib": args.c4_window_kib or 100, "counts": [int(x) for x in counts]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="harp", choices=("harp", "reference"))
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale of the workload (20 = the bench config)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-meter", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served-stream measurement")
    ap.add_argument("--workload", default="plain", choices=("plain", "partitioned", "whole"),
                    help="plain: the R-MAT bench; partitioned / whole: the Chung-Lu family of --n vertices, "
                         "partitioned under --cap-gib or counted whole on the device")
    ap.add_argument("--n", type=int, default=50_000_000, help="vertices of the Chung-Lu workloads")
    ap.add_argument("--cap-gib", type=float, default=24.0, help="device cap of the partitioned workload")
    ap.add_argument("--c4-window-kib", type=float, default=0,
                    help="whole workload: wedge window size of the plan (0 = the default 100 KiB)")
    ap.add_argument("--no-whole", action="store_true",
                    help="partitioned workload: skip the uncapped whole-graph count it is checked against")
    ap.add_argument("--no-partitioned", action="store_true",
                    help="skip the partitioned large-graph block of the default line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "partitioned":
        return run_partitioned(args)
    if args.workload == "whole":
        return run_whole(args)
    args.warmup = max(args.warmup, 3)

    world, rank, local = dist_env()
    import numpy as np
    import torch

    import graphgen
    from paper_2607_12074_gb300 import _build, harp, workmeter

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    harp.lib()

    g = graphgen.rmat(args.scale, 16, 0.57, 0.19, 0.19, seed=1)
    src_d = torch.from_numpy(g.src).cuda()
    dst_d = torch.from_numpy(g.dst).cuda()
    stream = torch.cuda.current_stream()
    csr = harp.harp_build_csr(g.n, src_d, dst_d, stream)
    info = csr.info()
    m = info["m"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    # ---- warm-up (also allocates and keeps the counting workspace)
    for _ in range(args.warmup):
        harp.harp_count4(csr)
    torch.cuda.synchronize()

    # ---- timed region: K steps, CUDA events on the launching stream, L2 flushed between steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    harp.harp_set_profiling(True)
    seg_ms = {k: [] for k in SEGMENTS}
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = harp.harp_launch_count()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.fill_(k)
            starts[k].record(stream)
            counts = harp.harp_count4(csr)
            ends[k].record(stream)
            ms, _ = harp.harp_last_stage_times()
            for name, v in zip(SEGMENTS, ms):
                seg_ms[name].append(v)
        torch.cuda.synchronize()
    launches = harp.harp_launch_count() - launches0
    harp.harp_set_profiling(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_step = sum(step_ms) / len(step_ms)
    t_step = max_over_ranks(t_step, world, "cuda")

    # ---- end to end through the public API from pinned host memory (build + count per step)
    src_h = torch.from_numpy(g.src).pin_memory()
    dst_h = torch.from_numpy(g.dst).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.fill_(k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g2 = harp.harp_build_csr(g.n, src_h.numpy(), dst_h.numpy(), stream)
        c2 = harp.harp_count4(g2)
        b.record(stream)
        torch.cuda.synchronize()
        g2.close()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
        assert np.array_equal(c2, counts)
    t_e2e = sum(e2e_ms) / len(e2e_ms)

    # the batched and served measurements are single-GPU workloads: skipped for replicas (N > 1)
    batched = None if (args.no_batched or world > 1) else bench_batched(harp, graphgen, np, torch, stream, flush,
                                                                        args.steps, args.warmup)
    served = None if (args.no_served or world > 1) else bench_served(harp, graphgen, np)
    # the partitioned large graph (one call, host edge list to counts, under the 24 GiB cap) and the
    # same graph counted whole: the owner rule's exactness check at full size
    partitioned = None if (args.no_partitioned or world > 1) else bench_partitioned(harp, graphgen, torch, args.n,
                                                                                      args.cap_gib)

    if rank != 0:
        return 0
    peak, peak_kind = load_peaks()
    seg_avg = {k: (sum(v) / len(v) if v else 0.0) for k, v in seg_ms.items()}
    roofline = None
    meter = None
    segment_rooflines = None
    if not args.no_meter:
        meter = workmeter.meter(g.n, g.src, g.dst)
        # every segment against the HBM roofline: its algorithmic bytes (work meter) over its CUDA-event
        # time; the windowed wedge kernel's per-window re-reads are listed apart as overhead
        segment_rooflines = {}
        for k in SEGMENTS:
            t_ms = seg_avg[k]
            alg_k = meter[k]["bytes"] if k in meter else 0
            if t_ms <= 0 or alg_k <= 0:
                continue
            ach = alg_k / (t_ms / 1000) / 1e9
            segment_rooflines[k] = {"ms": t_ms, "algorithmic_bytes": alg_k, "achieved_gbs": ach, "frac": ach / peak}
            if meter[k].get("overhead_bytes"):
                segment_rooflines[k]["overhead_bytes"] = meter[k]["overhead_bytes"]
        kernel_segments = [k for k in SEGMENTS if k != "orient"]
        dom = max(kernel_segments, key=lambda k: seg_avg[k])
        alg = meter[dom]["bytes"]
        achieved = alg / (seg_avg[dom] / 1000) / 1e9
        traffic = None
        tfile = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tfile):  # DRAM bytes of one ncu capture, valid while the kernel is unchanged
            import hashlib
            with open(tfile) as f:
                rec = json.load(f)
            src = os.path.join(ROOT, rec.get("source", ""))
            if dom in rec and os.path.isfile(src):
                with open(src, "rb") as f:
                    if hashlib.sha256(f.read()).hexdigest()[:16] == rec.get("source_sha256_16"):
                        traffic = rec[dom]
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                    "algorithmic_bytes": alg, "kernel_ms": seg_avg[dom],
                    "overhead_bytes": meter[dom].get("overhead_bytes", 0)}
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on the bench graph itself (R-MAT scale 20, the same generator call), all host cores
        r = oracle_sample_rate(args.scale, counts=True)
        cpu = {"value": r["m"] / r["seconds"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "cpu_model": host_cpu_model(),
               "sample": f"the whole bench graph: R-MAT scale {args.scale} (a,b,c = 0.57,0.19,0.19, ef 16, "
                         f"seed 1; m={r['m']}), oracle count4_combo (non-induced counts + inversion, OpenMP), "
                         f"one run of {r['seconds']:.1f} s",
               "counts_equal_gpu": [int(x) for x in counts] == r["counts"]}
        # Oracle A (the plain definition by ESU, one thread) on the plain small graph, against the GPU
        ra = oracle_a_rate()
        ga = graphgen.ba_2000()
        ca = harp.count4_edges(ga.n, ga.src, ga.dst)
        cpu["oracle_a"] = {"value": ra["m"] / ra["seconds"], "unit": UNIT, "threads": 1, "seconds": ra["seconds"],
                           "sample": f"Barabasi-Albert n=2000, 4 edges per new vertex, seed 1 (m={ra['m']}), "
                                     "oracle count4_esu (every connected 4-subset once, Wernicke's ESU)",
                           "counts_equal_gpu": [int(x) for x in ca] == ra["counts"]}
    value = replica_throughput(m, world, t_step)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"rmat(scale={args.scale}, ef=16, a=0.57, b=0.19, c=0.19, seed=1), symmetrised, "
                               f"self-loops and duplicates removed", "n": g.n, "m": m,
                   "max_degree": info["max_degree"], "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "flushed between steps (256 MiB write)"},
        "e2e": {"value": world * m / (t_e2e / 1000), "unit": UNIT, "h2d_bytes_per_step": 8 * g.m_in,
                "d2h_bytes_per_step": 72, "ms_per_step": t_e2e},
        "roofline": roofline,
        "segment_rooflines": segment_rooflines,
        "cpu_baseline": cpu,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "segments_ms": seg_avg,
        "batched": batched,
        "served": served,
        "partitioned": partitioned,
        "counts": [int(x) for x in counts],
        "hbm_pct_alg": (100.0 * sum(meter[k]["bytes"] for k in SEGMENTS) / (t_step / 1000) / 1e9 / peak)
        if meter else None,
    }
    print(json.dumps(line), flush=True)
    csr.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
