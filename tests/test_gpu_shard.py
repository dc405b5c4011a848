"""K row-block shards on one GPU: the shards of a build, run one after the
other, must reproduce the whole build.  The worklists of the shards are
disjoint and their union is the build's worklist (bit-exact); their
survivor counts add up exactly; the sum of their K equals the whole K and a
captured shard replays the eager shard.  In FP64 the only difference is the
order of the FP64 atomic adds (1e-12 relative).  In mixed precision the
FP32 partial sums of a warp depend on which records share the warp, which
differs between a shard and the whole build, so there the bar is the
contract's mixed-precision 1e-8.  The shards come from kx_row_work and
kx_shard_bounds (balanced ERI work)."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1401_6961_gb300 import build
    build.build()
    import paper_1401_6961_gb300 as kx
    kx.load()
    return kx


def _tol(opts, K):
    return 1e-8 if opts.get("precision", 0) == 1 else 1e-12 * max(1.0, K.abs().max().item())


def _sorted(w):
    w = np.asarray(w, dtype=np.int64).reshape(-1, 4)
    return w[np.lexsort(w.T[::-1])] if len(w) else w


CASES = [("water4", 4, dict(tau=1e-10)),
         ("water16", 16, dict(tau=1e-10)),
         ("water16", 16, dict(tau=1e-8, precision=1, split_threshold=5e-4))]


@pytest.mark.parametrize("symmetric", [0, 1])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_shards_reproduce_the_build(kx, case, symmetric):
    import torch
    from paper_1401_6961_gb300 import shard
    name, leaf_max, opts = CASES[case]
    sys_, P = wl.workload(name)
    opts = dict(opts, symmetric=symmetric)
    ex = kx.Exchange(sys_, leaf_max=leaf_max)
    Pd = torch.from_numpy(P).cuda()
    K0 = ex(Pd, keep_worklist=1, **opts).clone()
    st0 = ex.stats
    w0 = _sorted(ex.worklist())
    work = ex.row_work(Pd, **opts)
    full = ex.count(Pd, **opts)
    assert work.sum() == pytest.approx(full.flops_fp64 + full.flops_fp32, rel=1e-5)
    leaves, _ = ex.leaves()
    for n in (2, 3):
        b = shard.plan(ex, Pd, n, **opts)
        Ks = torch.zeros_like(K0)
        lists, nq = [], 0
        for r in range(n):
            so = shard.shard_opts(b, r, keep_worklist=1, **opts)
            Ks += ex(Pd, **so)
            nq += ex.stats.n_shell_quartets
            wr = ex.worklist()
            assert ((wr[:, 0] >= b[r]) & (wr[:, 0] < b[r + 1])).all()
            lists.append(wr)
            assert ex.count(Pd, **so).n_shell_quartets == ex.stats.n_shell_quartets
        torch.cuda.synchronize()
        assert nq == st0.n_shell_quartets
        assert np.array_equal(_sorted(np.concatenate(lists)), w0)
        assert (Ks - K0).abs().max().item() <= _tol(opts, K0)
    ex.close()


def test_captured_shard_replays_the_eager_shard(kx):
    import torch
    from paper_1401_6961_gb300 import shard
    sys_, P = wl.workload("water16")
    ex = kx.Exchange(sys_, leaf_max=16)
    Pd = torch.from_numpy(P).cuda()
    opts = dict(tau=1e-10, precision=1, split_threshold=5e-4, symmetric=1)
    b = shard.plan(ex, Pd, 2, **opts)
    so = shard.shard_opts(b, 1, **opts)
    Ke = ex(Pd, **so).clone()
    K = torch.empty_like(Pd)
    ex.plan(Pd, K, **so)
    ex.replay()
    torch.cuda.synchronize()
    assert (K - Ke).abs().max().item() <= _tol(opts, Ke)
    # and in FP64 to rounding order
    o64 = dict(opts, precision=0)
    so = shard.shard_opts(b, 1, **o64)
    Ke = ex(Pd, **so).clone()
    ex.plan(Pd, K, **so)
    ex.replay()
    torch.cuda.synchronize()
    assert (K - Ke).abs().max().item() <= _tol(o64, Ke)
    ex.close()


def test_shard_against_oracle_rows(kx):
    """One shard's rows (FP64) against the oracle's screened rows."""
    import torch
    from paper_1401_6961_gb300 import shard
    sys_, P = wl.workload("water4")
    ex = kx.Exchange(sys_, leaf_max=4)
    Pd = torch.from_numpy(P).cuda()
    b = shard.plan(ex, Pd, 2, tau=1e-10)
    K = ex(Pd, **shard.shard_opts(b, 0, tau=1e-10)).cpu().numpy()
    Kr, *_ = oracle.exchange_screened(sys_, P, 1e-10, leaf_max=4)
    leaves, _ = ex.leaves()
    order = ex.order()
    off = sys_.shell_offset
    rows = np.concatenate([np.arange(off[s], off[s + 1]) for s in order[leaves[b[0]][0]:leaves[b[1] - 1][1]]])
    assert np.abs(K[rows] - Kr[rows]).max() <= 1e-10
    other = np.setdiff1d(np.arange(sys_.n_fn), rows)
    assert np.abs(K[other]).max() == 0.0
    ex.close()


def test_bad_shard_ranges_are_rejected(kx):
    import torch
    sys_, P = wl.workload("water4")
    ex = kx.Exchange(sys_, leaf_max=4)
    Pd = torch.from_numpy(P).cuda()
    _, n_leaf = kx._binding._n_leaves(ex.ctx)
    for lo, hi in ((2, 2), (3, 1), (-1, 2), (0, n_leaf + 1)):
        with pytest.raises(kx.KxError) as e:
            ex(Pd, tau=1e-10, row_leaf_lo=lo, row_leaf_hi=hi)
        assert e.value.code == kx.KX_EINVAL
    ex.close()
