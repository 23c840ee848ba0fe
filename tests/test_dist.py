"""Multi-process aggregation of bench.py on CPU (gloo, world size 2).

Each rank of a replicated run times its own data set; the job's time is the
maximum over ranks and its throughput counts every rank's units.  The
reference-arm and non-zero ranks' rules are checked as host logic too.
"""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.dist_env()
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, w)
        value = bench.job_throughput(1000.0, w, job_ms * 1e-3)
        q.put((r, lr, w, job_ms, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, local, world, job_ms, value) in enumerate(res):
        assert (rank, local, world) == (r, r, 2)
        assert job_ms == 15.0                       # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 1000.0 / 0.015)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(10.0, 1, 2.0) == 5.0
