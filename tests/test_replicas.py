"""Whole-job timing of independent replicas across ranks (the bench's N>1
path), with two gloo processes on the CPU: every rank sees the slowest
rank's time, and the throughput counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2206_13932_gb300 import replicas
    ws, r = replicas.world()
    ms = replicas.max_over_ranks(10.0 + 5.0 * rank)          # rank 1 is slower
    thr = replicas.job_throughput(1000.0, ms)
    out.put((r, ws, ms, thr))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r, (rank, ws, ms, thr) in enumerate(got):
        assert rank == r and ws == 2
        assert ms == 15.0                                     # the slowest rank's time
        assert thr == pytest.approx(2 * 1000.0 / 15e-3)       # both ranks' units


def test_single_process_is_one_rank():
    from paper_2206_13932_gb300 import replicas
    assert replicas.world() == (1, 0)
    assert replicas.max_over_ranks(7.5) == 7.5
    assert replicas.job_throughput(100.0, 10.0) == pytest.approx(1e4)
