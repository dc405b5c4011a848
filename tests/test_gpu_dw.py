"""Double-word FP32 arithmetic for the quartets above the split
(KX_MIXED_DW): each value is an unevaluated sum of two floats, about 48
significant bits, computed on the FP32 pipe; classes with la+lb+lc+ld <= 5
have double-word kernels, the larger ones keep their FP64 kernels.

With split 0 every quartet of those classes runs in double words, and the
result must meet the FP64 contract (max|dK| <= 1e-10) against the oracle.
With the benchmark's split the FP32 bulk is unchanged, so the K must agree
with the plain mixed build to far below the mixed bar and meet the mixed
contract (1e-8) against the oracle's rows.
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


def test_all_double_word_water4_meets_the_fp64_bar(kx):
    sys_, P = wl.workload("water4")
    K0 = oracle.exchange_direct(sys_, P)
    for leaf_max in (4, 10):
        K, ex = _run(kx, sys_, P, leaf_max=leaf_max, tau=0.0, precision=kx.KX_MIXED_DW, split_threshold=0.0)
        st = ex.stats
        # s and p shells only: every class has a double-word kernel
        assert st.n_shell_quartets_dw == st.n_shell_quartets > 0 and st.n_shell_quartets_fp64 == 0
        assert np.abs(K - K0).max() <= TOL64
        ex.close()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_all_double_word_random_shells_all_classes(kx, seed):
    """d shells: the classes with la+lb+lc+ld >= 6 stay in FP64, the rest in
    double words; every class at the FP64 bar."""
    sys_ = wl.random_shells(9, seed, lmax=2, box=2.5)
    P = wl.density(sys_, 100 + seed)
    K0 = oracle.exchange_direct(sys_, P)
    for leaf_max in (1, 6):
        K, ex = _run(kx, sys_, P, leaf_max=leaf_max, tau=0.0, precision=kx.KX_MIXED_DW, split_threshold=0.0)
        st = ex.stats
        assert st.n_shell_quartets_dw > 0
        assert st.n_shell_quartets == st.n_shell_quartets_dw + st.n_shell_quartets_fp64
        assert np.abs(K - K0).max() <= TOL64
        ex.close()


def test_medium_waters_mixed_dw_against_oracle_and_mixed(kx):
    big = wl.water64(2)
    s3 = wl.build_system("w3", big.symbols[:9], big.xyz[:9] / wl.BOHR_PER_ANGSTROM, "medium")
    P = wl.density(s3, 3003)
    Kref, *_ = oracle.exchange_screened(s3, P, 1e-10)
    Kdw, ex = _run(kx, s3, P, tau=1e-10, precision=kx.KX_MIXED_DW, split_threshold=1e-4)
    st = ex.stats
    assert st.n_shell_quartets_dw > 0 and st.n_shell_quartets_fp64 > 0   # d shells: L >= 6 in FP64
    ex.close()
    Km, ex = _run(kx, s3, P, tau=1e-10, precision=kx.KX_MIXED, split_threshold=1e-4)
    assert ex.stats.n_shell_quartets == st.n_shell_quartets
    assert ex.stats.n_shell_quartets_fp64 == st.n_shell_quartets_fp64 + st.n_shell_quartets_dw
    ex.close()
    assert np.abs(Kdw - Kref).max() <= TOLMIX
    assert np.abs(Kdw - Km).max() <= 1e-10


def test_count_matches_the_double_word_build(kx):
    import torch
    sys_, P = wl.workload("water16")
    ex = kx.Exchange(sys_, leaf_max=16)
    Pd = torch.from_numpy(P).cuda()
    opts = dict(tau=1e-10, precision=kx.KX_MIXED_DW, split_threshold=5e-4, symmetric=1)
    ex(Pd, **opts)
    b = ex.stats
    c = ex.count(Pd, **opts)
    for f in ("n_shell_quartets", "n_shell_quartets_dw", "n_shell_quartets_fp64", "n_leaf_quartets"):
        assert getattr(c, f) == getattr(b, f), f
    assert c.flops_dw == pytest.approx(b.flops_dw, rel=1e-12) and b.flops_dw > 0
    ex.close()


def test_water64_mixed_dw_captured_rows(kx):
    """The benchmark system and launch configuration in KX_MIXED_DW: sampled
    rows (two of them d shells) against the oracle at the mixed bar, and
    the whole K against the plain mixed build of the same split."""
    import torch
    sys_, P = wl.workload("water64")
    ex = kx.Exchange(sys_, leaf_max=16)
    Pd = torch.from_numpy(P).cuda()
    Kd = torch.empty_like(Pd)
    opts = dict(tau=1e-10, precision=kx.KX_MIXED_DW, split_threshold=5e-4, symmetric=1)
    ex.autotune(Pd, out=Kd, **opts)
    ex.plan(Pd, Kd, **opts)
    Kd.zero_()
    ex.replay()
    torch.cuda.synchronize()
    assert ex.stats.n_shell_quartets_dw > 0
    K = Kd.cpu().numpy()
    # (the eager build chunks its leaves differently, so its FP32 warp sums
    # differ: the mixed bar)
    Km = ex(Pd, tau=1e-10, precision=kx.KX_MIXED, split_threshold=5e-4, symmetric=1).cpu().numpy()
    assert np.abs(K - Km).max() <= TOLMIX
    L = np.asarray(sys_.shell_l)
    rng = np.random.default_rng(66)
    rows = [int(x) for x in rng.choice(np.nonzero(L == 2)[0], 2, replace=False)]
    rows += [int(x) for x in rng.choice(np.nonzero(L < 2)[0], 2, replace=False)]
    Kref, *_ = oracle.exchange_screened(sys_, P, 1e-10, leaf_max=16, rows=rows)
    off = sys_.shell_offset
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
    assert np.abs(K[idx] - Kref[idx]).max() <= TOLMIX
    ex.close()
