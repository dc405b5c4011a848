"""Symmetric builds (kx_opts.symmetric = 1): for a symmetric P the exchange
matrix is symmetric, K_{nu mu} = sum (nu lam|mu sig) P_{lam sig} = K_{mu nu}
by the bra-ket symmetry (mu lam|nu sig) = (nu sig|mu lam) of Eq. 6's
integrals, so only the K blocks (A,C) with A <= C (tree order) are built and
the others are mirrored.  The result must still equal the oracle's full sum,
and the worklist must be the oracle's worklist restricted to A <= C.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-8


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


def _run(kx, sys_, P, leaf_max=10, **opts):
    import torch
    ex = kx.Exchange(sys_, leaf_max=leaf_max)
    K = ex(torch.from_numpy(np.ascontiguousarray(P)).cuda(), **opts)
    torch.cuda.synchronize()
    return K.cpu().numpy(), ex


def _sorted(w):
    w = np.asarray(w, dtype=np.int64).reshape(-1, 4)
    return w[np.lexsort(w.T[::-1])] if len(w) else w


def test_water4_symmetric_tau0_and_screened(kx):
    sys_, P = wl.workload("water4")
    K0 = oracle.exchange_direct(sys_, P)
    K, ex = _run(kx, sys_, P, tau=0.0, symmetric=1)
    assert np.abs(K - K0).max() <= TOL64
    ex.close()
    for tau in (1e-10, 1e-6):
        Kref, wref, nq, tree, s2 = oracle.exchange_screened(sys_, P, tau)
        K, ex = _run(kx, sys_, P, tau=tau, symmetric=1, keep_worklist=1)
        assert np.abs(K - Kref).max() <= TOL64
        w = ex.worklist()
        half = wref[wref[:, 0] <= wref[:, 2]]
        assert np.array_equal(_sorted(w), _sorted(half))
        ex.close()


@pytest.mark.parametrize("leaf_max", [1, 6])
def test_random_shells_symmetric(kx, leaf_max):
    sys_ = wl.random_shells(10, 77)
    P = wl.density(sys_, 78)
    K0 = oracle.exchange_direct(sys_, P)
    K, ex = _run(kx, sys_, P, leaf_max=leaf_max, tau=0.0, symmetric=1)
    assert np.abs(K - K0).max() <= TOL64
    ex.close()


def test_medium_basis_symmetric_halves_the_work(kx):
    s = wl.water_cluster(3, 7, "medium")
    P = wl.density(s, 1007)
    Kref, *_ = oracle.exchange_screened(s, P, 1e-10)
    Kf, exf = _run(kx, s, P, tau=1e-10)
    nfull = exf.stats.n_shell_quartets
    K, ex = _run(kx, s, P, tau=1e-10, symmetric=1)
    nsym = ex.stats.n_shell_quartets
    assert np.abs(K - Kref).max() <= TOL64
    assert np.abs(K - K.T).max() <= 1e-12
    # a <= c of every (a,c): half of the off-diagonal blocks plus the diagonal
    assert nfull / 2 <= nsym < 0.6 * nfull
    Km, exm = _run(kx, s, P, tau=1e-10, symmetric=1, precision=kx.KX_MIXED, split_threshold=1e-4)
    assert np.abs(Km - Kref).max() <= TOLMIX
    for e in (exf, ex, exm):
        e.close()


def test_batch_symmetric_and_graph(kx):
    import torch
    systems = [wl.water_cluster(n, 800 + n, "small") for n in (2, 4, 6)] + [wl.water_cluster(2, 9, "medium")]
    dens = [wl.density(s, 3000 + i) for i, s in enumerate(systems)]
    bx = kx.BatchExchange(systems)
    P = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).cuda()
    Ke = bx(P, tau=1e-8, symmetric=1).clone()
    for y, (s, d) in enumerate(zip(systems, dens)):
        Kref, *_ = oracle.exchange_screened(s, d, 1e-8)
        got = Ke[bx.offsets[y]:bx.offsets[y + 1]].cpu().numpy().reshape(Kref.shape)
        assert np.abs(got - Kref).max() <= TOL64, s.name
    K = torch.empty_like(P)
    bx.plan(P, K, tau=1e-8, symmetric=1, precision=kx.KX_MIXED, split_threshold=1e-4)
    K.zero_()
    bx.replay()
    torch.cuda.synchronize()
    assert torch.abs(K - Ke).max().item() <= TOLMIX
    bx.close()


BENCH_LEAF = 16   # bisection leaf size of the benchmark builds


def test_water64_symmetric_mixed_rows(kx):
    """The benchmark system in the benchmark's launch configuration (leaf
    size 16, tuned shapes, captured build replayed, double words above the
    split, the split planned from an 8e-9 FP32 budget, symmetric): 16
    sampled K-row shells (4 d, 6 p, 6 s) against the oracle at the same leaf
    size, and the leaf worklist of those rows against the oracle's
    traversal."""
    import torch
    sys_, P = wl.workload("water64")
    ex = kx.Exchange(sys_, leaf_max=BENCH_LEAF)
    Pd = torch.from_numpy(P).cuda()
    Kd = torch.empty_like(Pd)
    sp = ex.split_plan(Pd, 8e-9, tau=1e-10, symmetric=1)
    assert sp.split_used > 0
    opts = dict(tau=1e-10, precision=kx.KX_MIXED_DW, split_threshold=sp.split_used, symmetric=1)
    ex.autotune(Pd, out=Kd, **opts)
    ex.plan(Pd, Kd, **opts)
    Kd.zero_()
    ex.replay()
    torch.cuda.synchronize()
    K = Kd.cpu().numpy()
    L = np.asarray(sys_.shell_l)
    rng = np.random.default_rng(65)
    rows = [int(x) for l, k in ((2, 4), (1, 6), (0, 6)) for x in rng.choice(np.nonzero(L == l)[0], k, replace=False)]
    Kref, wref, nq, tree, s2 = oracle.exchange_screened(sys_, P, 1e-10, leaf_max=BENCH_LEAF, rows=rows)
    off = sys_.shell_offset
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
    assert np.abs(K[idx] - Kref[idx]).max() <= TOLMIX
    # the mirrored half: columns of the same rows
    assert np.abs(K[:, idx] - Kref[idx].T).max() <= TOLMIX
    # the worklist of an eager build of the same configuration, restricted to
    # the leaves that hold the sampled rows: the oracle's, with A <= C
    ex(Pd, out=Kd, keep_worklist=1, **opts)
    leaves, _ = ex.leaves()
    pos = {int(s): i for i, s in enumerate(ex.order())}
    aleaf = sorted({int(np.searchsorted(leaves[:, 1], pos[r], side="right")) for r in rows})
    w = ex.worklist(aleaf)
    half = wref[wref[:, 0] <= wref[:, 2]]
    assert set(half[:, 0].tolist()) <= set(aleaf)
    assert np.array_equal(_sorted(w), _sorted(half))
    ex.close()
