"""Pins of the oracle's exchange build, ordering, tree and traversal.

* Exchange (Eq. 6 without -1/2): one-hot P reproduces single integrals,
  K = K^T, linearity, permutation covariance, block-diagonal K for far
  fragments.
* Hilbert order: unit steps along the whole curve on an 8^3 grid, and the
  two neighbours of random cells on the 1024^3 grid.
* Ragged bisection (Eq. 1): the split rule checked by brute force.
* Traversal (Eqs. 7, 8): equals brute-force enumeration of every leaf
  quartet whose own bound exceeds tau (child norms never exceed parent
  norms, so hierarchical culling removes exactly those).
* tau = 0: the screened method equals the plain definition.
* tau > 0: the error obeys the rigorous bound of Eq. 8.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import workloads as wl

NC = (1, 3, 6)


@pytest.fixture(scope="module")
def w4():
    s = wl.water4(1)
    return s, wl.density(s, 1001)


@pytest.fixture(scope="module")
def w2():
    """(H2O)_2 with the small basis: a quick direct-exchange case."""
    rng = np.random.default_rng(21)
    syms, xyz = wl._place_waters(np.array([[0.0, 0, 0], [2.9, 0.3, 0.1]]), rng)
    s = wl.build_system("(H2O)2", syms, xyz, "small")
    return s, wl.density(s, 2021)


@pytest.fixture(scope="module")
def w3med():
    """Three waters from the (H2O)_64 cluster with the medium basis (d shells)."""
    big = wl.water64(2)
    keep_atoms = list(range(9))
    syms = [big.symbols[i] for i in keep_atoms]
    s = wl.build_system("(H2O)3m", syms, big.xyz[keep_atoms] / wl.BOHR_PER_ANGSTROM, "medium")
    return s, wl.density(s, 3003)


# ---------------------------------------------------------------------------
# exchange definition
# ---------------------------------------------------------------------------

def test_onehot_density_gives_integrals(w2):
    s, _ = w2
    off = s.shell_offset
    rng = np.random.default_rng(0)
    for _ in range(3):
        b, d = rng.integers(0, s.n_shell, size=2)
        j = rng.integers(0, NC[s.shell_l[b]])
        l = rng.integers(0, NC[s.shell_l[d]])
        P = np.zeros((s.n_fn, s.n_fn))
        P[off[b] + j, off[d] + l] = 1.0
        K = oracle.exchange_direct(s, P)
        for a in range(s.n_shell):
            for c in range(s.n_shell):
                ctr = s.xyz[s.shell_atom]
                v = oracle.eri(ctr[a], s.shell_alpha[a], s.shell_l[a], ctr[b], s.shell_alpha[b], s.shell_l[b],
                               ctr[c], s.shell_alpha[c], s.shell_l[c], ctr[d], s.shell_alpha[d], s.shell_l[d])
                np.testing.assert_allclose(K[off[a]:off[a + 1], off[c]:off[c + 1]], v[:, j, :, l],
                                           rtol=1e-13, atol=1e-15)


def test_exchange_symmetric_and_linear(w2):
    s, P = w2
    K = oracle.exchange_direct(s, P)
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    rng = np.random.default_rng(1)
    Q = rng.standard_normal(P.shape)
    Q = Q + Q.T
    KQ = oracle.exchange_direct(s, Q)
    K2 = oracle.exchange_direct(s, 2.5 * P - 0.75 * Q)
    np.testing.assert_allclose(K2, 2.5 * K - 0.75 * KQ, rtol=0, atol=1e-12 * np.abs(K2).max())


def test_exchange_nonsymmetric_P_gives_transpose(w2):
    # K(P^T) = K(P)^T by (mu lam|nu sig) = (nu sig|mu lam)
    s, _ = w2
    rng = np.random.default_rng(2)
    P = rng.standard_normal((s.n_fn, s.n_fn))
    K = oracle.exchange_direct(s, P)
    KT = oracle.exchange_direct(s, P.T.copy())
    np.testing.assert_allclose(KT, K.T, rtol=0, atol=1e-12 * np.abs(K).max())


def test_exchange_permutation_covariance(w2):
    s, P = w2
    K = oracle.exchange_direct(s, P)
    rng = np.random.default_rng(3)
    sp_ = rng.permutation(s.n_shell)
    s2 = wl.System(s.name, s.symbols, s.xyz, s.shell_atom[sp_], s.shell_l[sp_], s.shell_alpha[sp_])
    off = s.shell_offset
    fperm = np.concatenate([np.arange(off[i], off[i + 1]) for i in sp_])
    K2 = oracle.exchange_direct(s2, P[np.ix_(fperm, fperm)])
    np.testing.assert_allclose(K2, K[np.ix_(fperm, fperm)], rtol=0, atol=1e-13 * np.abs(K).max())


def test_exchange_far_fragments_block_diagonal():
    rng = np.random.default_rng(4)
    syms, xyz = wl._place_waters(np.array([[0.0, 0, 0], [60.0, 0, 0]]), rng)
    s = wl.build_system("far", syms, xyz, "small")
    n1 = s.n_fn // 2
    P = wl.density(s, 44)
    P[:n1, n1:] = 0.0
    P[n1:, :n1] = 0.0
    K = oracle.exchange_direct(s, P)
    assert np.abs(K[:n1, n1:]).max() < 1e-200
    assert np.abs(K[:n1, :n1]).max() > 1e-2


# ---------------------------------------------------------------------------
# Hilbert order
# ---------------------------------------------------------------------------

def test_hilbert_full_grid_unit_steps():
    bits = 3
    n = 1 << bits
    cells = list(itertools.product(range(n), repeat=3))
    keys = np.array([oracle.key_of_cell(c, bits) for c in cells])
    assert sorted(keys.tolist()) == list(range(n ** 3))
    order = np.argsort(keys)
    path = np.array(cells)[order]
    steps = np.abs(np.diff(path, axis=0)).sum(axis=1)
    assert np.all(steps == 1)


def test_hilbert_10bit_neighbours():
    rng = np.random.default_rng(5)
    for _ in range(200):
        q = rng.integers(1, 1023, size=3)
        k = oracle.key_of_cell(q, 10)
        nk = []
        for ax in range(3):
            for dlt in (-1, 1):
                r = q.copy()
                r[ax] += dlt
                nk.append(oracle.key_of_cell(r, 10))
        # the curve enters and leaves every interior cell through a face
        assert (k - 1) in nk and (k + 1) in nk


def test_shell_order_is_atom_major_hilbert(w4):
    s, _ = w4
    perm = oracle.shell_order(s)
    assert sorted(perm.tolist()) == list(range(s.n_shell))
    keys = oracle.hilbert_keys(s.xyz)
    atoms = s.shell_atom[perm]
    # atoms appear in contiguous runs ordered by (key, index)
    runs = [a for i, a in enumerate(atoms) if i == 0 or atoms[i - 1] != a]
    assert len(runs) == s.n_atom
    assert runs == sorted(runs, key=lambda a: (keys[a], a))
    for a in range(s.n_atom):
        sh = perm[atoms == a]
        assert np.all(np.diff(sh) > 0)


# ---------------------------------------------------------------------------
# bisection (Eq. 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("leaf_max", [1, 4, 10, 16])
def test_tree_split_rule(leaf_max):
    rng = np.random.default_rng(leaf_max)
    ls = rng.integers(0, 3, size=57).astype(np.int32)
    s = wl.System("t", ["X"] * 57, np.zeros((57, 3)), np.arange(57, dtype=np.int32), ls,
                  np.ones(57))
    perm = np.arange(57, dtype=np.int32)
    t = oracle.tree_build(s, leaf_max, perm)
    nfn = np.array([NC[x] for x in ls])
    pre = np.concatenate([[0], np.cumsum(nfn)])
    leaves = 0
    for v in range(t.n_node):
        lo, hi = t.lo[v], t.hi[v]
        f = pre[hi] - pre[lo]
        if t.child0[v] < 0:
            leaves += 1
            assert f <= leaf_max or hi - lo == 1
            continue
        assert f > leaf_max and hi - lo > 1
        c0, c1 = t.child0[v], t.child1[v]
        assert t.lo[c0] == lo and t.hi[c1] == hi and t.hi[c0] == t.lo[c1]
        cand = range(lo + 1, hi)
        best = min(cand, key=lambda x: (abs(2 * pre[x] - pre[lo] - pre[hi]), x))
        assert t.hi[c0] == best
    assert leaves == t.n_leaf
    lr = t.leaf_ranges()
    assert lr[0, 0] == 0 and lr[-1, 1] == 57 and np.all(lr[1:, 0] == lr[:-1, 1])


# ---------------------------------------------------------------------------
# traversal (Eqs. 7, 8) and the screened build
# ---------------------------------------------------------------------------

def _sorted(w):
    w = np.asarray(w).reshape(-1, 4)
    if len(w) == 0:
        return w
    return w[np.lexsort(w.T[::-1])]


@pytest.mark.parametrize("tau", [0.0, 1e-6, 1e-3, 3e-2])
@pytest.mark.parametrize("leaf_max", [4, 10])
def test_traversal_equals_bruteforce(w4, tau, leaf_max):
    s, P = w4
    tree = oracle.tree_build(s, leaf_max)
    s2 = oracle.schwarz_sq(s)
    work = oracle.traverse(s, P, tree, s2, tau)
    brute, beta = oracle.leaf_bruteforce(s, P, tree, s2, tau)
    a, b = _sorted(work), _sorted(brute)
    if len(a) != len(b) or not np.array_equal(a, b):
        # only threshold-grazing items may differ (the norm sums are
        # evaluated in different orders at different levels)
        sa = {tuple(x) for x in a}
        sb = {tuple(x) for x in b}
        allq, allb = oracle.leaf_bruteforce(s, P, tree, s2, -1.0)
        bmap = {tuple(q): v for q, v in zip(allq, allb)}
        for q in sa ^ sb:
            assert abs(bmap[q] - tau) <= 1e-13 * max(tau, 1e-300), q
    assert len(a) > 0


def test_traversal_medium_basis(w3med):
    s, P = w3med
    tree = oracle.tree_build(s, 10)
    s2 = oracle.schwarz_sq(s)
    for tau in (1e-8, 1e-4):
        work = oracle.traverse(s, P, tree, s2, tau)
        brute, _ = oracle.leaf_bruteforce(s, P, tree, s2, tau)
        assert np.array_equal(_sorted(work), _sorted(brute))


@pytest.mark.parametrize("shell_screen", [False, True])
@pytest.mark.parametrize("leaf_max", [4, 10, 1000])
def test_tau_zero_equals_direct(w4, shell_screen, leaf_max):
    s, P = w4
    K0 = oracle.exchange_direct(s, P)
    K, work, nq, tree, s2 = oracle.exchange_screened(s, P, 0.0, leaf_max, shell_screen)
    np.testing.assert_allclose(K, K0, rtol=0, atol=1e-13 * np.abs(K0).max())


def test_tau_zero_equals_direct_medium(w3med):
    s, P = w3med
    K0 = oracle.exchange_direct(s, P)
    K, *_ = oracle.exchange_screened(s, P, 0.0, 10, True)
    np.testing.assert_allclose(K, K0, rtol=0, atol=1e-13 * np.abs(K0).max())


@pytest.mark.parametrize("tau", [1e-5, 1e-3])
def test_culling_error_within_rigorous_bound(w4, tau):
    s, P = w4
    K0 = oracle.exchange_direct(s, P)
    tree = oracle.tree_build(s, 10)
    s2 = oracle.schwarz_sq(s)
    allq, allb = oracle.leaf_bruteforce(s, P, tree, s2, -1.0)
    work = oracle.traverse(s, P, tree, s2, tau)
    kept = {tuple(x) for x in work}
    bound_leaf = sum(b for q, b in zip(allq, allb) if tuple(q) not in kept)
    # without the shell screen: only whole leaf quartets are dropped
    K1, _ = oracle.exchange_worklist(s, P, tree, s2, tau, work, shell_screen=False)
    err1 = np.linalg.norm(K1 - K0)
    assert 0 < err1 <= bound_leaf
    # with it: add the shell quartets screened inside kept leaves
    K2, _ = oracle.exchange_worklist(s, P, tree, s2, tau, work, shell_screen=True)
    pq = oracle.pblock_sq(s, P)
    S, Pn = np.sqrt(s2), np.sqrt(pq)
    lr = tree.leaf_ranges()
    extra = 0.0
    for q in work:
        A, B, C, D = [tree.perm[lr[x, 0]:lr[x, 1]] for x in q]
        b = (S[np.ix_(A, B)][:, :, None, None] * Pn[np.ix_(B, D)][None, :, None, :]) * S[np.ix_(C, D)][None, None]
        extra += b[b <= tau].sum()
    err2 = np.linalg.norm(K2 - K0)
    assert err2 <= bound_leaf + extra


def test_row_sampled_equals_full_rows(w4):
    s, P = w4
    K, *_ = oracle.exchange_screened(s, P, 1e-10)
    rows = [0, 5, 17, 30]
    Kr, *_ = oracle.exchange_screened(s, P, 1e-10, rows=rows)
    off = s.shell_offset
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
    np.testing.assert_allclose(Kr[idx], K[idx], rtol=0, atol=1e-14 * np.abs(K).max())
    mask = np.ones(s.n_fn, bool)
    mask[idx] = False
    assert np.all(Kr[mask] == 0)


def test_overlap_pruning_eq4(w4):
    s, P = w4
    tau_ovlp = 1e-3
    s2 = oracle.schwarz_sq(s, tau_ovlp)
    ctr = s.xyz[s.shell_atom]
    pruned = 0
    for a in range(s.n_shell):
        for b in range(s.n_shell):
            ov = oracle.overlap(ctr[a], s.shell_alpha[a], s.shell_l[a], ctr[b], s.shell_alpha[b], s.shell_l[b])
            if s2[a, b] == 0.0:
                pruned += 1
                assert np.abs(ov).max() < tau_ovlp
            else:
                assert np.abs(ov).max() >= tau_ovlp
    assert pruned > 0
