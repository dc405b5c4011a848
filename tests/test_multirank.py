"""The benchmark's multi-rank path on CPU: world size 2 over gloo.

Every rank builds its own K (replicas), so the only cross-rank steps are the
barrier around the timed region and the maximum of the ranks' times; the job
value counts every rank's builds over the slowest rank's time.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        bench.barrier(ws)
        # rank r "took" 1.5 + r seconds for its two builds
        slowest = bench.max_over_ranks(1.5 + rank, ws, "cpu")
        bench.barrier(ws)
        out[rank] = (env, slowest, bench.job_rate(2, ws, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_aggregation_over_gloo():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(90)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(ws):
        env, slowest, rate = res[r]
        assert env == (ws, r, r)
        assert slowest == 2.5                 # max over ranks
        assert rate == pytest.approx(2 * 2 / 2.5)   # all ranks' builds / slowest time


def test_single_rank_is_a_no_op():
    bench.barrier(1)
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_rate(256, 1, 2.0) == 128.0
