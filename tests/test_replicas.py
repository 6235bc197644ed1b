"""Replicas on several GPUs (the path shards across independent problems): the
bench's barrier, its maximum of the timed region over ranks, the disjoint
per-rank inputs and the whole-job value, run as two gloo ranks on the CPU; the
reference arm prints on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.replica_barrier(world)
        # a slower rank 1: the job's time is the slowest rank's
        local_ms = 100.0 + 50.0 * rank
        job_ms = bench.replica_max(local_ms, world, torch.device("cpu"))
        seeds = bench.replica_seeds(rank, 8)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out.put((rank, job_ms, bench.whole_job_value(8, world, 5, job_ms), gathered))
        bench.replica_barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_and_value_over_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job_ms, value, gathered in res:
        assert job_ms == 150.0
        assert value == pytest.approx(8 * 2 * 5 / 0.150)
        assert not set(gathered[0]) & set(gathered[1])


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.reference_arm(A(), 1) is None
    assert capsys.readouterr().out == ""
