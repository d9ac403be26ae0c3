"""The bench's multi-rank path on CPU (gloo, world size 2): every rank times
its own replica, the job's timed region is the slowest rank's (all-reduce
MAX), the whole-job value counts the units of all ranks, and only rank 0
reports.  A single system does not shard, so there is no data-path
collective to test beyond this."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, loc = bench.dist_env()
        local_ms = 100.0 + 37.0 * rank  # rank 1 is the slow one
        job_ms = bench.reduce_max_ms(local_ms, w)
        value = bench.job_value(5.0e6, job_ms / 10, w)  # 10 steps
        out.put((r, w, loc, job_ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, ws, local, job_ms, value) in enumerate(res):
        assert (rank, ws, local) == (r, 2, r)
        assert job_ms == 137.0  # max over ranks
        assert value == pytest.approx(2 * 5.0e6 / (137.0e-3 / 10))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_ms(12.5, 1) == 12.5
    assert bench.job_value(10.0, 2.0, 1) == pytest.approx(5000.0)
