"""The multi-GPU path of the benchmark is replicas only (the solver has no
exchange step): every rank runs the same workload, the job time is the
slowest rank's, and the reported throughput counts the DoFs of all ranks.
Checked with two gloo ranks on the CPU."""
import os

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.job_rate(100.0 + 50.0 * rank, 10, 1000, world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_counts_all_ranks():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, value = res[r]
        assert ms == pytest.approx(15.0)                     # max(100, 150) ms / 10 steps
        assert value == pytest.approx(2 * 1000 / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.job_rate(80.0, 8, 500, 1)
    assert ms == pytest.approx(10.0) and value == pytest.approx(500 / 10e-3 / 1e9)
