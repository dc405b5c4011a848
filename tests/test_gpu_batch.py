"""Batched exchange: many independent systems in one context (kx_create_batch).

Every system of a batch is an independent problem (Eqs. 6-8 per system), so
each system's block of the packed K must match the oracle run on that system
alone: max |dK| <= 1e-10 in FP64 and <= 1e-8 in mixed precision, and the
system's part of the forest worklist (leaf ordinals shifted to the system's
own tree) must equal the oracle's traversal of that system.
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


def _one_shell():
    return wl.System(name="one_shell", symbols=["X"], xyz=np.zeros((1, 3)),
                     shell_atom=np.zeros(1, dtype=np.int32), shell_l=np.zeros(1, dtype=np.int32),
                     shell_alpha=np.array([0.7]))


@pytest.fixture(scope="module")
def small_batch():
    """Uneven systems: 1..5 waters (small basis), 3 waters with d shells,
    one single shell, all-class random shells."""
    systems = [wl.water_cluster(n, 900 + n, "small") for n in (1, 2, 3, 5)]
    systems += [wl.water_cluster(3, 7, "medium"), _one_shell(), wl.random_shells(9, 31)]
    dens = [wl.density(s, 2000 + i) for i, s in enumerate(systems)]
    return systems, dens


def _run(kx, systems, dens, **opts):
    import torch
    bx = kx.BatchExchange(systems)
    P = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).cuda()
    K = bx(P, **opts)
    torch.cuda.synchronize()
    Ks = [k.cpu().numpy() for k in bx.unpack(K)]
    return Ks, bx


def _sorted(w):
    w = np.asarray(w, dtype=np.int64).reshape(-1, 4)
    return w[np.lexsort(w.T[::-1])] if len(w) else w


def _split_worklist(bx, work):
    """Per system: its quartets with leaf ordinals of its own tree."""
    leaves, _ = bx.leaves()
    sys_of_leaf = np.searchsorted(bx.shell_offsets, leaves[:, 0], side="right") - 1
    first = np.searchsorted(sys_of_leaf, np.arange(bx.n_sys))
    out = []
    ys = sys_of_leaf[work[:, 0]] if len(work) else np.zeros(0, dtype=np.int64)
    for y in range(bx.n_sys):
        w = work[ys == y]
        assert np.all(sys_of_leaf[w] == y), "a quartet mixes systems"
        out.append(w - first[y])
    return out, sys_of_leaf, first


def test_order_and_trees_per_system(kx, small_batch):
    systems, dens = small_batch
    _, bx = _run(kx, systems, dens, tau=1e-8)
    order = bx.order()
    leaves, _ = bx.leaves()
    for y, s in enumerate(systems):
        o0 = bx.shell_offsets[y]
        assert np.array_equal(order[o0:o0 + s.n_shell] - o0, oracle.shell_order(s))
        t = oracle.tree_build(s, 10)
        mine = leaves[(leaves[:, 0] >= o0) & (leaves[:, 0] < o0 + s.n_shell)] - o0
        assert np.array_equal(mine, t.leaf_ranges())


def test_norm_blocks_match_oracle(kx, small_batch):
    systems, dens = small_batch
    _, bx = _run(kx, systems, dens, tau=1e-8)
    total = int(sum(s.n_shell ** 2 for s in systems))
    s2, pq = kx.kx_get_norms(bx.ctx, 0, True, total=total)
    off = 0
    for s, P in zip(systems, dens):
        n = s.n_shell
        ref = oracle.schwarz_sq(s)
        mine = s2[off:off + n * n].reshape(n, n)
        rel = np.abs(mine - ref) / np.maximum(np.abs(ref), 1e-300)
        k = np.unravel_index(np.argmax(rel), rel.shape)
        # McMurchie-Davidson (library) and Obara-Saika (oracle) round
        # differently; the random shells (d shells, exponents 0.1..8, short
        # distances) reach 1.1e-12 relative, the water blocks stay <= 1e-13
        tol = 1e-11 if s.name.startswith("random") else 1e-13
        assert rel.max() <= tol, (s.name, float(rel.max()), float(ref[k]), float(mine[k]), k)
        assert np.array_equal(pq[off:off + n * n].reshape(n, n), oracle.pblock_sq(s, P))
        off += n * n


def test_batch_tau0_equals_direct(kx, small_batch):
    systems, dens = small_batch
    Ks, _ = _run(kx, systems, dens, tau=0.0)
    for s, P, K in zip(systems, dens, Ks):
        K0 = oracle.exchange_direct(s, P)
        assert np.abs(K - K0).max() <= TOL64, s.name


@pytest.mark.parametrize("tau", [1e-8, 1e-4])
def test_batch_screened_fp64_and_worklists(kx, small_batch, tau):
    systems, dens = small_batch
    Ks, bx = _run(kx, systems, dens, tau=tau, keep_worklist=1)
    parts, _, _ = _split_worklist(bx, bx.worklist())
    for s, P, K, w in zip(systems, dens, Ks, parts):
        Kref, wref, nq, tree, s2 = oracle.exchange_screened(s, P, tau)
        assert np.abs(K - Kref).max() <= TOL64, s.name
        assert np.array_equal(_sorted(w), _sorted(wref)), s.name


def test_batch_mixed(kx, small_batch):
    systems, dens = small_batch
    Ks, _ = _run(kx, systems, dens, tau=1e-8, precision=kx.KX_MIXED, split_threshold=1e-4)
    for s, P, K in zip(systems, dens, Ks):
        Kref, *_ = oracle.exchange_screened(s, P, 1e-8)
        assert np.abs(K - Kref).max() <= TOLMIX, s.name


def test_batch_equals_single_contexts(kx, small_batch):
    """Packing changes nothing: each block equals a single-system build."""
    import torch
    systems, dens = small_batch
    Ks, bx = _run(kx, systems, dens, tau=1e-8, keep_worklist=1)
    parts, _, _ = _split_worklist(bx, bx.worklist())
    for s, P, K, w in zip(systems, dens, Ks, parts):
        ex = kx.Exchange(s)
        K1 = ex(torch.from_numpy(P).cuda(), tau=1e-8, keep_worklist=1).cpu().numpy()
        assert np.abs(K - K1).max() <= 1e-12
        assert np.array_equal(_sorted(w), _sorted(ex.worklist()))
        ex.close()


def test_batch_host_entry_point(kx, small_batch):
    systems, dens = small_batch
    Ks, bx = _run(kx, systems, dens, tau=1e-8)
    Kh = bx.host(np.concatenate([d.ravel() for d in dens]), tau=1e-8)
    for y, K in enumerate(Ks):
        o0, o1 = bx.offsets[y], bx.offsets[y + 1]
        assert np.abs(Kh[o0:o1].reshape(K.shape) - K).max() <= 1e-12


def test_batch_argument_errors(kx, small_batch):
    import torch
    systems, dens = small_batch
    bx = kx.BatchExchange(systems[:2])
    P = torch.zeros(bx.size, dtype=torch.float64, device="cuda")
    with pytest.raises(kx.KxError) as e:
        kx.kx_exchange(bx.ctx, P.data_ptr(), 1, kx.kx_default_opts(), P.data_ptr(), 1)
    assert e.value.code == kx.KX_EINVAL
    with pytest.raises(kx.KxError) as e:
        kx.kx_traverse(bx.ctx, P.data_ptr(), 1, kx.kx_default_opts())
    assert e.value.code == kx.KX_ENOTIMPL
    with pytest.raises(kx.KxError) as e:
        kx.kx_create_batch([])
    assert e.value.code == kx.KX_EINVAL
    bx.close()


# ---------------------------------------------------------------------------
# the full batched workload (256 clusters of 4..48 waters, tau = 1e-8, mixed
# precision), in the launch configuration of the benchmark: sampled systems
# against the oracle, K rows of sampled shells
# ---------------------------------------------------------------------------

def test_batch256_sampled_systems(kx):
    """Launch configuration of the benchmark: tuned shapes, captured build
    replayed, split 5e-4, symmetric builds."""
    import torch
    systems, dens = wl.batch_workload()
    bx = kx.BatchExchange(systems)
    P = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).cuda()
    K = torch.empty_like(P)
    opts = dict(tau=1e-8, precision=kx.KX_MIXED, split_threshold=5e-4, symmetric=1)
    bx.autotune(P, out=K, **opts)
    bx.plan(P, K, **opts)
    K.zero_()
    bx.replay()
    torch.cuda.synchronize()
    Ks = bx.unpack(K)
    nf = np.array([s.n_fn for s in systems])
    picks = [int(np.argmin(nf)), int(np.argsort(nf)[len(nf) // 2]), int(np.argmax(nf))]
    rng = np.random.default_rng(256)
    for y in picks:
        s = systems[y]
        rows = sorted(rng.choice(s.n_shell, size=min(3, s.n_shell), replace=False).tolist())
        Kref, *_ = oracle.exchange_screened(s, dens[y], 1e-8, rows=rows)
        off = s.shell_offset
        fr = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
        got = Ks[y].cpu().numpy()[fr]
        assert np.abs(got - Kref[fr]).max() <= TOLMIX, (y, s.n_fn)
    bx.close()


# ---------------------------------------------------------------------------
# captured builds (CUDA graph replay) and the launch-shape autotuner
# ---------------------------------------------------------------------------

def test_graph_replay_matches_eager(kx, small_batch):
    import torch
    systems, dens = small_batch
    bx = kx.BatchExchange(systems)
    P = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).cuda()
    Ke = bx(P, tau=1e-8).clone()
    ste = bx.stats
    K = torch.empty_like(P)
    bx.plan(P, K, headroom=0.25, tau=1e-8)
    assert torch.abs(K - Ke).max().item() <= 1e-12
    K.zero_()
    bx.replay()
    torch.cuda.synchronize()
    assert torch.abs(K - Ke).max().item() <= 1e-12
    assert bx.stats.n_shell_quartets == ste.n_shell_quartets
    assert bx.stats.n_leaf_quartets == ste.n_leaf_quartets
    # new contents of the captured P: a slightly different density
    dens2 = [0.9 * d for d in dens]
    P.copy_(torch.from_numpy(np.concatenate([d.ravel() for d in dens2])))
    bx.replay()
    torch.cuda.synchronize()
    for y, (s, d) in enumerate(zip(systems, dens2)):
        Kref, *_ = oracle.exchange_screened(s, d, 1e-8)
        got = K[bx.offsets[y]:bx.offsets[y + 1]].cpu().numpy().reshape(Kref.shape)
        assert np.abs(got - Kref).max() <= TOL64, s.name
    bx.close()


def test_graph_replay_mixed(kx, small_batch):
    import torch
    systems, dens = small_batch
    bx = kx.BatchExchange(systems)
    P = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).cuda()
    K = torch.empty_like(P)
    bx.plan(P, K, tau=1e-8, precision=kx.KX_MIXED, split_threshold=1e-4)
    K.zero_()
    bx.replay()
    torch.cuda.synchronize()
    for y, (s, d) in enumerate(zip(systems, dens)):
        Kref, *_ = oracle.exchange_screened(s, d, 1e-8)
        got = K[bx.offsets[y]:bx.offsets[y + 1]].cpu().numpy().reshape(Kref.shape)
        assert np.abs(got - Kref).max() <= TOLMIX, s.name
    bx.close()


def test_graph_overflow_is_reported(kx, small_batch):
    """A replay that needs more than the plan reserved stops at its
    capacity checks and reports KX_ECAPACITY; a new plan then works."""
    import torch
    systems, dens = small_batch
    bx = kx.BatchExchange(systems)
    P = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).cuda()
    K = torch.empty_like(P)
    bx.plan(P, K, headroom=0.0, tau=1e-4)
    P.mul_(1e3)          # larger ||P|| blocks: many more quartets survive
    with pytest.raises(kx.KxError) as e:
        bx.replay()
    assert e.value.code == kx.KX_ECAPACITY
    bx.plan(P, K, headroom=0.0, tau=1e-4)
    Ke = K.clone()
    K.zero_()
    bx.replay()
    torch.cuda.synchronize()
    assert torch.abs(K - Ke).max().item() <= 1e-12 * max(1.0, Ke.abs().max().item())
    bx.close()


def test_autotune_keeps_results(kx, small_batch):
    import torch
    systems, dens = small_batch
    systems = systems + [wl.water_cluster(12, 12, "small")]
    dens = dens + [wl.density(systems[-1], 2012)]
    bx = kx.BatchExchange(systems)
    P = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).cuda()
    Ke = bx(P, tau=1e-10).clone()
    Kt = bx.autotune(P, tau=1e-10)
    assert bx.n_tuned >= 1
    threads, bpsm, variant = kx.kx_get_launch_shapes(bx.ctx)
    assert set(threads.tolist()) <= {64, 128, 256} and (bpsm >= 0).all()
    K2 = bx(P, tau=1e-10)
    torch.cuda.synchronize()
    assert torch.abs(Kt - Ke).max().item() <= 1e-12
    assert torch.abs(K2 - Ke).max().item() <= 1e-12
    bx.close()
