"""The multi-GPU path of the benchmark is replicas only: each rank counts its
own corpus, with no exchange on the data path; ranks meet only for the
timing barrier and the max-over-ranks step time.  That host logic runs here
as two gloo ranks on the CPU (no GPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # the second rank is the slow one
        dist.barrier()
        m = bench.max_over_ranks(ms, dist, "cpu")
        q.put((rank, m, bench.job_rate(1000.0, world, m), bench.replica_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_the_slowest_and_count_every_rank():
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    assert all(g[1] == 15.0 for g in got)                      # max over ranks
    assert all(g[2] == pytest.approx(1000.0 * 2 / 0.015) for g in got)  # all ranks' units / slowest time
    assert got[0][3] != got[1][3]                              # each replica its own corpus


def test_one_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_rate(2e9, 1, 4.0) == pytest.approx(5e11)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 3

    # rank 1 of 2 returns at once, without building or running the oracle
    assert bench.run_reference(Args(), 1, 2) is None
