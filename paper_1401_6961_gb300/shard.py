"""K row-block shards across ranks: one GPU per rank, each building the K
rows of its leaves (kx_opts.row_leaf_lo/hi), then one sum of the partial K
matrices over the ranks (every entry comes from exactly one shard, so the
sum is an exact assembly).  The shards come from kx_row_work and
kx_shard_bounds: contiguous leaf ranges of balanced ERI work."""
from __future__ import annotations

from typing import Tuple

import numpy as np

from . import _binding as kb


def plan(ex, P, n_shards: int, **opts) -> np.ndarray:
    """Leaf boundaries of n_shards balanced row-block shards of the build
    ``ex(P, **opts)``."""
    work = ex.row_work(P, **opts)
    return kb.kx_shard_bounds(work, n_shards)


def rows_of(bounds, rank: int) -> Tuple[int, int]:
    """The leaf range [lo, hi) of shard `rank`."""
    return int(bounds[rank]), int(bounds[rank + 1])


def shard_opts(bounds, rank: int, **opts) -> dict:
    lo, hi = rows_of(bounds, rank)
    return dict(opts, row_leaf_lo=lo, row_leaf_hi=hi)


def assemble(K, group=None):
    """Sum the ranks' partial K in place (one all-reduce); returns K."""
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(K, op=dist.ReduceOp.SUM, group=group)
    return K
