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


# ---------------------------------------------------------------------------
# K row-block shards: assignment (kx_shard_bounds, host code of the C ABI)
# and assembly (one sum over the ranks), world size 2 and 3 over gloo
# ---------------------------------------------------------------------------

def _fake_build(bounds, rank, leaf_fn, K_full, symmetric):
    """The partial K a shard writes: its rows, and in a symmetric build the
    lower triangle left out and mirrored from its rows (leaf_fn: function
    range of every leaf, in tree order = function order here)."""
    import numpy as np
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    f0, f1 = leaf_fn[lo][0], leaf_fn[hi - 1][1]
    K = np.zeros_like(K_full)
    if not symmetric:
        K[f0:f1] = K_full[f0:f1]
    else:
        # blocks (A, C) with A <= C for A in the shard, then their mirror
        K[f0:f1, f0:] = K_full[f0:f1, f0:]
        K[f0:, f0:f1] = K[f0:f1, f0:].T
    return K


def _shard_rank(rank: int, ws: int, port: int, out):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import paper_1401_6961_gb300 as kx
        from paper_1401_6961_gb300 import shard
        rng = np.random.default_rng(5)
        n_leaf = 13
        sizes = rng.integers(3, 9, size=n_leaf)
        edges = np.concatenate([[0], np.cumsum(sizes)])
        leaf_fn = [(int(edges[i]), int(edges[i + 1])) for i in range(n_leaf)]
        work = rng.random(n_leaf) * 10
        bounds = kx.kx_shard_bounds(work, ws)     # every rank computes the same plan
        res = {"bounds": bounds.tolist()}
        for symmetric in (0, 1):
            A = rng.standard_normal((edges[-1], edges[-1]))
            K_full = A + A.T if symmetric else A
            Kp = torch.from_numpy(_fake_build(bounds, rank, leaf_fn, K_full, symmetric))
            shard.assemble(Kp)
            res[f"err{symmetric}"] = float(np.abs(Kp.numpy() - K_full).max())
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("ws", [2, 3])
def test_row_block_shards_assemble_over_gloo(ws):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_shard_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(150)
            assert p.exitcode == 0
        res = dict(out)
    b = res[0]["bounds"]
    assert all(res[r]["bounds"] == b for r in range(ws))
    assert b[0] == 0 and b[-1] == 13 and all(b[i] < b[i + 1] for i in range(ws))
    for r in range(ws):
        assert res[r]["err0"] == 0.0 and res[r]["err1"] == 0.0


def test_shard_bounds_cover_balance_and_reject():
    import numpy as np
    import paper_1401_6961_gb300 as kx
    rng = np.random.default_rng(9)
    for n_leaf in (1, 2, 7, 50, 300):
        w = rng.random(n_leaf) ** 3 * 100
        for n in range(1, min(n_leaf, 9) + 1):
            b = kx.kx_shard_bounds(w, n)
            assert b[0] == 0 and b[-1] == n_leaf and (np.diff(b) >= 1).all()
            loads = [w[b[i]:b[i + 1]].sum() for i in range(n)]
            # each boundary is the nearest leaf boundary to its target, so no
            # shard exceeds the mean by more than the two largest leaves
            assert max(loads) <= w.sum() / n + 2 * w.max() + 1e-9
    assert (kx.kx_shard_bounds(np.zeros(6), 3) == [0, 2, 4, 6]).all()
    for bad in [(np.ones(3), 4), (np.ones(3), 0), (np.array([1.0, -1.0]), 1), (np.array([np.nan]), 1)]:
        with pytest.raises(kx.KxError):
            kx.kx_shard_bounds(*bad)
