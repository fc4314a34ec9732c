"""The multi-rank path of bench.py on the CPU (gloo, two ranks).

With N ranks each answering the same batch (replicas), the job's time is the
slowest rank's (a max over the ranks that every rank receives) and its
throughput counts every rank's queries; under a multi-rank launch the
reference arm works on rank 0 only and the other ranks return at once.
"""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms = b.max_over_ranks(1.0 + rank, world, "cpu")  # rank r took r + 1 ms
    out[rank] = (ms, b.job_throughput(world, 10_000, ms / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_and_whole_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        got = dict(out)
    assert got[0] == got[1] == (2.0, 2 * 10_000 / 2e-3)


def test_single_rank_keeps_its_own_time():
    b = _bench()
    assert b.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert b.job_throughput(1, 10, 0.5) == 20.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:  # no workload, no oracle: rank 1 must not touch either
        pass

    assert b.run_reference(Args()) == 0
