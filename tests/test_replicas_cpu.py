"""The replicated multi-GPU bench path, checked on the CPU with the gloo backend (world size 2): the
job's step time is the slowest rank's and its throughput counts every replica's edges."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [12.5, 30.25][rank]
    got = bench.max_over_ranks(local, world, "cpu")
    out[rank] = (got, bench.replica_throughput(15_702_112, world, got))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 30.25
    assert res[0][1] == res[1][1] == pytest.approx(2 * 15_702_112 / 0.03025)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(7.0, 1, "cpu") == 7.0
    assert bench.replica_throughput(1000, 1, 2.0) == pytest.approx(500_000.0)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        warmup, steps, gpus = 1, 1, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
