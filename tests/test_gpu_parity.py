"""Parity of the CUDA library (called through its C ABI) with the CPU oracle.

Tolerances (from the contract of the build): max |dK| <= 1e-10 in FP64
mode, <= 1e-8 in mixed mode; the leaf-quartet worklist must equal the
oracle's traversal except for quartets whose bound grazes tau (both sides
evaluate the same FP64 products on norms that differ by a few ulps, see
`_assert_same_worklist`).
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


def _gpu_k(kx, sys_, P, leaf_max=10, perm=None, tau_ovlp=0.0, **opts):
    import torch
    ex = kx.Exchange(sys_, leaf_max=leaf_max, perm=perm, tau_ovlp=tau_ovlp)
    Pd = torch.from_numpy(np.ascontiguousarray(P)).cuda()
    K = ex(Pd, **opts)
    torch.cuda.synchronize()
    return K.cpu().numpy(), ex


def _sorted(w):
    w = np.asarray(w, dtype=np.int64).reshape(-1, 4)
    return w[np.lexsort(w.T[::-1])] if len(w) else w


def _assert_same_worklist(gpu, ref, sys_, P, tree, s2, tau):
    a, b = _sorted(gpu), _sorted(ref)
    if len(a) == len(b) and np.array_equal(a, b):
        return
    sa, sb = {tuple(x) for x in a}, {tuple(x) for x in b}
    diff = sa ^ sb
    allq, allb = oracle.leaf_bruteforce(sys_, P, tree, s2, -1.0)
    beta = {tuple(q): v for q, v in zip(allq, allb)}
    bad = [q for q in diff if abs(beta[q] - tau) > 1e-12 * max(tau, 1e-300)]
    assert not bad, f"{len(bad)} non-grazing worklist differences, e.g. {bad[:5]}"


# ---------------------------------------------------------------------------
# order, tree, norms
# ---------------------------------------------------------------------------

def test_order_and_leaves_match_oracle(kx):
    for sys_ in (wl.water4(1), wl.water64(2)):
        ex = kx.Exchange(sys_)
        assert np.array_equal(ex.order(), oracle.shell_order(sys_))
        leaves, depth = ex.leaves()
        t = oracle.tree_build(sys_, 10)
        assert np.array_equal(leaves, t.leaf_ranges())
        assert depth == int(t.depth.max())
        ex.close()


def test_norm_tables_match_oracle(kx):
    sys_, P = wl.workload("water4")
    K, ex = _gpu_k(kx, sys_, P, tau=1e-10)
    s2, pq = ex.norms()
    ref_s2 = oracle.schwarz_sq(sys_)
    np.testing.assert_allclose(s2, ref_s2, rtol=1e-13, atol=1e-300)
    # same bytes of P, same summation order: identical
    assert np.array_equal(pq, oracle.pblock_sq(sys_, P))


def test_overlap_prune_matches_oracle(kx):
    sys_, P = wl.workload("water4")
    import torch
    ex = kx.Exchange(sys_, tau_ovlp=1e-3)
    s2, _ = ex.norms(with_p=False)
    ref = oracle.schwarz_sq(sys_, 1e-3)
    assert np.array_equal(s2 == 0, ref == 0)
    np.testing.assert_allclose(s2, ref, rtol=1e-13, atol=1e-300)


# ---------------------------------------------------------------------------
# (H2O)_4, 52 functions: tau = 0 against the plain definition, 1e-10 against
# the screened oracle, worklists against the oracle's traversal
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def w4_ref():
    sys_, P = wl.workload("water4")
    return sys_, P, oracle.exchange_direct(sys_, P)


@pytest.mark.parametrize("shell_screen", [1, 0])
def test_water4_tau0_equals_direct(kx, w4_ref, shell_screen):
    sys_, P, K0 = w4_ref
    K, ex = _gpu_k(kx, sys_, P, tau=0.0, shell_screen=shell_screen, keep_worklist=1)
    assert np.abs(K - K0).max() <= TOL64
    t = oracle.tree_build(sys_, 10)
    assert len(ex.worklist()) == t.n_leaf ** 4


@pytest.mark.parametrize("tau", [1e-10, 1e-6, 1e-3])
@pytest.mark.parametrize("leaf_max", [4, 10])
def test_water4_screened(kx, tau, leaf_max):
    sys_, P = wl.workload("water4")
    Kref, work, nq, tree, s2 = oracle.exchange_screened(sys_, P, tau, leaf_max)
    K, ex = _gpu_k(kx, sys_, P, leaf_max=leaf_max, tau=tau, keep_worklist=1)
    assert np.abs(K - Kref).max() <= TOL64
    _assert_same_worklist(ex.worklist(), work, sys_, P, tree, s2, tau)
    assert ex.stats.n_shell_quartets == nq


def test_water4_mixed(kx, w4_ref):
    sys_, P, K0 = w4_ref
    Kref, *_ = oracle.exchange_screened(sys_, P, 1e-10)
    K, ex = _gpu_k(kx, sys_, P, tau=1e-10, precision=kx.KX_MIXED, split_threshold=1e-4)
    assert ex.stats.n_shell_quartets_fp64 < ex.stats.n_shell_quartets
    assert np.abs(K - Kref).max() <= TOLMIX


# ---------------------------------------------------------------------------
# every angular-momentum class, d shells, ragged trees
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_shells_all_classes(kx, seed):
    sys_ = wl.random_shells(9, seed, lmax=2, box=2.5)
    assert set(sys_.shell_l.tolist()) == {0, 1, 2} or seed > 1
    P = wl.density(sys_, 100 + seed)
    K0 = oracle.exchange_direct(sys_, P)
    for leaf_max in (1, 6):
        K, ex = _gpu_k(kx, sys_, P, leaf_max=leaf_max, tau=0.0)
        err = np.abs(K - K0).max()
        print(f"seed {seed} leaf {leaf_max}: max|dK| {err:.2e}, max|K| {np.abs(K0).max():.2f}")
        assert err <= TOL64


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_shells_all_classes_fp32(kx, seed):
    """Every class through its FP32 kernel (split above every bound): the
    error is FP32 rounding of the integrals, bounded relative to max|K|."""
    sys_ = wl.random_shells(9, seed, lmax=2, box=2.5)
    P = wl.density(sys_, 100 + seed)
    K0 = oracle.exchange_direct(sys_, P)
    K, ex = _gpu_k(kx, sys_, P, leaf_max=6, tau=0.0, precision=kx.KX_MIXED, split_threshold=1e30)
    assert ex.stats.n_shell_quartets_fp64 == 0
    assert np.abs(K - K0).max() <= 2e-5 * np.abs(K0).max()


@pytest.mark.parametrize("seed", [1, 2])
def test_random_shells_fp32_pruned_variant(kx, seed):
    """The FP32 large classes through their ket-pruned kernel, forced for
    every such class (split above every bound: all quartets in FP32)."""
    sys_ = wl.random_shells(9, seed, lmax=2, box=2.5)
    P = wl.density(sys_, 100 + seed)
    K0 = oracle.exchange_direct(sys_, P)
    import torch
    ex = kx.Exchange(sys_, leaf_max=6)
    big = [81 + c for c in range(81) if c // 27 + c // 9 % 3 + c // 3 % 3 + c % 3 >= 7]
    for s in big:
        kx.kx_set_launch_shape(ex.ctx, s, 128, 0, 1)
    assert kx.kx_get_launch_shapes(ex.ctx)[2][big].tolist() == [1] * len(big)
    with pytest.raises(kx.KxError):
        kx.kx_set_launch_shape(ex.ctx, big[0], 128, 0, 2)   # two kernels per FP32 large class
    K = ex(torch.from_numpy(P).cuda(), tau=0.0, precision=kx.KX_MIXED, split_threshold=1e30).cpu().numpy()
    assert ex.stats.n_shell_quartets_fp64 == 0
    assert np.abs(K - K0).max() <= 2e-5 * np.abs(K0).max()
    ex.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("seed", [1, 2])
def test_random_shells_fp64_shared_memory_variant(kx, seed, variant):
    """The FP64 large classes through their other kernels (shared-memory R
    with full Hermite sets; the same with the ket set pruned per nu), forced
    for every such class."""
    sys_ = wl.random_shells(9, seed, lmax=2, box=2.5)
    P = wl.density(sys_, 100 + seed)
    K0 = oracle.exchange_direct(sys_, P)
    import torch
    ex = kx.Exchange(sys_, leaf_max=6)
    big = [c for c in range(81) if c // 27 + c // 9 % 3 + c // 3 % 3 + c % 3 >= 7]
    for c in big:
        kx.kx_set_launch_shape(ex.ctx, c, 128, 0, variant)
    assert kx.kx_get_launch_shapes(ex.ctx)[2][big].tolist() == [variant] * len(big)
    with pytest.raises(kx.KxError):
        kx.kx_set_launch_shape(ex.ctx, big[0], 128, 0, 3)   # three kernels per FP64 large class
    with pytest.raises(kx.KxError):
        kx.kx_set_launch_shape(ex.ctx, 0, 128, 0, 1)      # (ss|ss) has one kernel
    K = ex(torch.from_numpy(P).cuda(), tau=0.0).cpu().numpy()
    assert np.abs(K - K0).max() <= TOL64
    ex.close()


@pytest.mark.parametrize("opts", [dict(), dict(symmetric=1), dict(shell_screen=0),
                                  dict(precision=1, split_threshold=1e-4),
                                  dict(precision=1, split_threshold=1e-4, symmetric=1)])
def test_count_equals_build_and_oracle(kx, opts):
    """kx_count reports the survivors of the build it stands for without
    building K: the same counts as the build, and (every K block, shell
    screen on) the oracle's leaf worklist length and shell-quartet count."""
    import torch
    big = wl.water64(2)
    w3 = wl.build_system("w3", big.symbols[:9], big.xyz[:9] / wl.BOHR_PER_ANGSTROM, "medium")
    for sys_, P in (wl.workload("water4"), (w3, wl.density(w3, 3003))):
        for tau in (1e-10, 1e-6):
            ex = kx.Exchange(sys_)
            Pd = torch.from_numpy(np.ascontiguousarray(P)).cuda()
            c = ex.count(Pd, tau=tau, **opts)
            ex(Pd, tau=tau, **opts)
            b = ex.stats
            assert c.n_leaf_quartets == b.n_leaf_quartets > 0
            assert c.n_shell_quartets == b.n_shell_quartets > 0
            assert c.n_shell_quartets_fp64 == b.n_shell_quartets_fp64
            assert c.n_candidates == b.n_candidates
            assert c.depth == b.depth and list(c.n_tasks) == list(b.n_tasks)
            assert c.flops_fp64 == pytest.approx(b.flops_fp64, rel=1e-12)
            assert c.flops_fp32 == pytest.approx(b.flops_fp32, rel=1e-12)
            if not opts.get("symmetric") and opts.get("shell_screen", 1):
                _, work, nq, _, _ = oracle.exchange_screened(sys_, P, tau)
                assert c.n_leaf_quartets == len(work)
                assert c.n_shell_quartets == nq
            ex.close()


def test_medium_basis_three_waters(kx):
    big = wl.water64(2)
    s = wl.build_system("w3", big.symbols[:9], big.xyz[:9] / wl.BOHR_PER_ANGSTROM, "medium")
    P = wl.density(s, 3003)
    K0 = oracle.exchange_direct(s, P)
    K, ex = _gpu_k(kx, s, P, tau=0.0)
    assert np.abs(K - K0).max() <= TOL64
    Kref, work, nq, tree, s2 = oracle.exchange_screened(s, P, 1e-10)
    K, ex = _gpu_k(kx, s, P, tau=1e-10, keep_worklist=1)
    assert np.abs(K - Kref).max() <= TOL64
    _assert_same_worklist(ex.worklist(), work, s, P, tree, s2, 1e-10)
    Km, ex = _gpu_k(kx, s, P, tau=1e-10, precision=kx.KX_MIXED, split_threshold=1e-4)
    assert np.abs(Km - Kref).max() <= TOLMIX


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_single_shell_system(kx):
    s = wl.System("one", ["X"], np.zeros((1, 3)), np.array([0], np.int32), np.array([2], np.int32),
                  np.array([0.7]))
    P = wl.density(s, 5)
    K0 = oracle.exchange_direct(s, P)
    K, ex = _gpu_k(kx, s, P, tau=0.0)
    assert ex.stats.depth == 0
    assert np.abs(K - K0).max() <= TOL64


def test_everything_culled_gives_zero(kx):
    sys_, P = wl.workload("water4")
    K, ex = _gpu_k(kx, sys_, P, tau=1e6)
    assert ex.stats.n_leaf_quartets == 0 and np.all(K == 0)


def test_nonsymmetric_P_and_padded_leading_dims(kx):
    import torch
    sys_, _ = wl.workload("water4")
    rng = np.random.default_rng(7)
    n = sys_.n_fn
    P = rng.standard_normal((n, n))
    K0 = oracle.exchange_direct(sys_, P)
    ex = kx.Exchange(sys_)
    Pp = torch.zeros((n, n + 5), dtype=torch.float64, device="cuda")
    Pp[:, :n] = torch.from_numpy(P).cuda()
    Kp = torch.full((n, n + 3), 7.0, dtype=torch.float64, device="cuda")
    o = kx.kx_default_opts(tau=0.0)
    kx.kx_exchange(ex.ctx, Pp.data_ptr(), n + 5, o, Kp.data_ptr(), n + 3)
    torch.cuda.synchronize()
    Kh = Kp.cpu().numpy()
    assert np.abs(Kh[:, :n] - K0).max() <= TOL64
    assert np.all(Kh[:, n:] == 7.0)


def test_host_entry_point_matches_device(kx, w4_ref):
    sys_, P, K0 = w4_ref
    ex = kx.Exchange(sys_)
    Kh = ex.host(P, tau=0.0)
    assert np.abs(Kh - K0).max() <= TOL64


def test_explicit_permutation(kx, w4_ref):
    sys_, P, K0 = w4_ref
    perm = np.random.default_rng(3).permutation(sys_.n_shell).astype(np.int32)
    K, ex = _gpu_k(kx, sys_, P, perm=perm, tau=0.0)
    assert np.array_equal(ex.order(), perm)
    assert np.abs(K - K0).max() <= TOL64


def test_small_chunks_give_same_K(kx):
    sys_, P = wl.workload("water4")
    K1, _ = _gpu_k(kx, sys_, P, tau=1e-10)
    K2, ex = _gpu_k(kx, sys_, P, tau=1e-10, chunk_records=5000)
    assert ex.stats.n_chunks > 1
    assert np.abs(K1 - K2).max() <= 1e-13


def test_call_order_and_argument_errors(kx):
    sys_, P = wl.workload("water4")
    ctx = kx.kx_create(sys_.xyz, sys_.shell_atom, sys_.shell_l, sys_.shell_alpha)
    import torch
    Pd = torch.from_numpy(P).cuda()
    K = torch.empty_like(Pd)
    with pytest.raises(kx.KxError) as e:
        kx.kx_exchange(ctx, Pd.data_ptr(), sys_.n_fn, kx.kx_default_opts(), K.data_ptr(), sys_.n_fn)
    assert e.value.code == kx.KX_ESTATE
    with pytest.raises(kx.KxError) as e:
        kx.kx_build_tree(ctx, 10)
    assert e.value.code == kx.KX_ESTATE
    kx.kx_build_schwarz(ctx)
    kx.kx_build_tree(ctx, 10)
    for bad in (dict(tau=-1.0), dict(precision=7), dict(tau=float("nan"))):
        with pytest.raises(kx.KxError) as e:
            kx.kx_exchange(ctx, Pd.data_ptr(), sys_.n_fn, kx.kx_default_opts(**bad), K.data_ptr(), sys_.n_fn)
        assert e.value.code == kx.KX_EINVAL
    with pytest.raises(kx.KxError) as e:
        kx.kx_exchange(ctx, Pd.data_ptr(), sys_.n_fn - 1, kx.kx_default_opts(), K.data_ptr(), sys_.n_fn)
    assert e.value.code == kx.KX_EINVAL
    with pytest.raises(kx.KxError) as e:
        kx.kx_build_tree(ctx, 10, perm=[0] * sys_.n_shell)
    assert e.value.code == kx.KX_EINVAL
    kx.kx_destroy(ctx)


# ---------------------------------------------------------------------------
# (H2O)_64, 1984 functions, tau = 1e-10: the benchmark workload.  K rows of
# sampled shells against the oracle's row-restricted traversal and
# contraction; the worklist restricted to the leaves holding those shells.
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def w64(kx):
    import torch
    sys_, P = wl.workload("water64")
    ex = kx.Exchange(sys_)
    Pd = torch.from_numpy(P).cuda()
    K64 = ex(Pd, tau=1e-10, keep_worklist=1).cpu().numpy()
    st64 = ex.stats
    rows = [int(x) for x in np.random.default_rng(64).choice(sys_.n_shell, size=3, replace=False)]
    rows.append(int(np.nonzero(sys_.shell_l == 2)[0][5]))
    leaves, _ = ex.leaves()
    order = ex.order()
    pos = {int(s): i for i, s in enumerate(order)}
    aleaf = sorted({int(np.searchsorted(leaves[:, 1], pos[r], side="right")) for r in rows})
    work = ex.worklist(aleaf)
    Km = ex(Pd, tau=1e-10, precision=kx.KX_MIXED, split_threshold=1e-4).cpu().numpy()
    stm = ex.stats
    Kref, wref, nq, tree, s2 = oracle.exchange_screened(sys_, P, 1e-10, rows=rows)
    ex.close()
    return sys_, P, rows, K64, st64, Km, stm, Kref, work, wref, aleaf, tree, s2


def test_water64_fp64_rows(w64):
    sys_, P, rows, K64, st64, Km, stm, Kref, work, wref, aleaf, tree, s2 = w64
    off = sys_.shell_offset
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
    assert np.abs(K64[idx] - Kref[idx]).max() <= TOL64
    assert st64.n_leaf_quartets > 0 and st64.n_shell_quartets > 0


def test_water64_worklist_rows(w64):
    sys_, P, rows, K64, st64, Km, stm, Kref, work, wref, aleaf, tree, s2 = w64
    a = _sorted(work)
    b = _sorted(wref)
    assert set(a[:, 0].tolist()) <= set(aleaf)
    assert np.array_equal(a, b)


def test_water64_mixed_rows(w64):
    sys_, P, rows, K64, st64, Km, stm, Kref, work, wref, aleaf, tree, s2 = w64
    off = sys_.shell_offset
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
    assert np.abs(Km[idx] - Kref[idx]).max() <= TOLMIX
    assert np.abs(Km - K64).max() <= TOLMIX
    assert stm.n_shell_quartets == st64.n_shell_quartets


def test_sweep_member_water128_mixed_rows(kx):
    """A member of the (H2O)_n scaling sweep, (H2O)_128 (3968 functions),
    tau = 1e-8, built as the benchmark builds (mixed, split 5e-4,
    symmetric): sampled K-row shells (one of them d) against the oracle."""
    import torch
    sys_ = wl.water_sweep(128, "medium")
    P = wl.density(sys_, 5128)
    ex = kx.Exchange(sys_)
    Pd = torch.from_numpy(P).cuda()
    K = ex(Pd, tau=1e-8, precision=kx.KX_MIXED, split_threshold=5e-4, symmetric=1).cpu().numpy()
    assert ex.stats.n_shell_quartets_fp64 > 0
    ex.close()
    rows = [int(np.random.default_rng(128).integers(sys_.n_shell)), int(np.nonzero(sys_.shell_l == 2)[0][17])]
    Kref, *_ = oracle.exchange_screened(sys_, P, 1e-8, rows=rows)
    off = sys_.shell_offset
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
    assert np.abs(K[idx] - Kref[idx]).max() <= TOLMIX
    # symmetric build: the mirrored columns agree as well
    assert np.abs(K[:, idx] - Kref[idx].T).max() <= TOLMIX
