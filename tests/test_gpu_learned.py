"""Learned culling on the GPU: the library's training kernels against the
FP64 reference network, and what the trained network gains over the plain
Schwarz x ||P|| culling at the same tau, with the error it adds judged
against the exact traversal."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import mlp

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


def _rand(seed, n=300):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.25, mlp.NP).astype(np.float32)
    p[mlp.P_MU:mlp.P_IS] = rng.normal(0, 1, mlp.NF)
    p[mlp.P_IS:mlp.P_W1] = np.abs(rng.normal(0.5, 0.1, mlp.NF))
    X = rng.normal(0, 2, (n, mlp.NF)).astype(np.float32)
    T = rng.normal(-8, 2, n).astype(np.float32)
    return p, X, T


def test_gpu_gradient_matches_reference(kx):
    import torch
    p, X, T = _rand(1, 333)
    pd, Xd, Td = (torch.from_numpy(a).cuda() for a in (p, X, T))
    g = torch.zeros_like(pd)
    loss = kx.kx_mlp_loss_grad(pd.data_ptr(), Xd.data_ptr(), Td.data_ptr(), X.shape[0], g.data_ptr())
    ref_loss, ref_g = mlp.loss_grad(p.astype(np.float64), X, T)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    gg = g.cpu().numpy()
    assert np.all(gg[:mlp.P_W1] == 0)
    scale = np.abs(ref_g).max()
    assert np.abs(gg - ref_g).max() <= 2e-4 * scale


def test_gpu_bf16_inference_matches_reference(kx):
    import torch
    p, X, _ = _rand(2, 1000)
    pd, Xd = torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()
    out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    kx.kx_mlp_infer_bf16(pd.data_ptr(), Xd.data_ptr(), X.shape[0], out.data_ptr())
    torch.cuda.synchronize()
    ref, _ = mlp.forward(p.astype(np.float64), X)
    err = np.abs(out.cpu().numpy() - ref)
    # BF16 operands (8-bit significand) through three layers
    assert err.max() <= 0.05 * (1 + np.abs(ref).max())
    assert np.median(err) <= 0.01 * (1 + np.abs(ref).max())


def test_gpu_adam_matches_reference(kx):
    import torch
    p, X, T = _rand(3)
    rng = np.random.default_rng(5)
    g = rng.normal(0, 1e-2, mlp.NP).astype(np.float32)
    m = rng.normal(0, 1e-3, mlp.NP).astype(np.float32)
    v = np.abs(rng.normal(0, 1e-4, mlp.NP)).astype(np.float32)
    pd, gd, md, vd = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    kx.kx_mlp_adam(pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), 1e-3, 7)
    rp, rm, rv = mlp.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                          1e-3, 7)
    np.testing.assert_allclose(pd.cpu().numpy(), rp, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(md.cpu().numpy(), rm, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(vd.cpu().numpy(), rv, rtol=1e-5, atol=1e-12)


@pytest.fixture(scope="module")
def trained(kx):
    """The network trained on water clusters (configurations 1 and 3: two
    small clusters and two clusters of the batched workload) and its cull
    margin calibrated on alkanes, a family kept out of training: the 99.9 %
    quantile of how far the true contribution lies above the prediction."""
    import torch
    from paper_1401_6961_gb300 import learned
    tau = 1e-8

    def tr_of(sys_, P):
        ex = kx.Exchange(sys_)
        t = learned.traces(ex, torch.from_numpy(P).cuda(), tau, max_samples=12000, seed=1)
        ex.close()
        return t
    w8 = wl.water_cluster(8, 8, "small")
    bs, bd = wl.batch_workload(count=4)
    tr = None
    for sys_, P in (wl.workload("water4"), (w8, wl.density(w8, 808)), (bs[0], bd[0]), (bs[1], bd[1])):
        t = tr_of(sys_, P)
        tr = t if tr is None else tr + t
    model = learned.train(tr, epochs=300, lr=3e-3, batch=4096)
    c6, c10 = wl.alkane(6, 66), wl.alkane(10, 610)
    held = tr_of(c6, wl.density(c6, 812)) + tr_of(c10, wl.density(c10, 7610))
    model = learned.calibrate(model, held, q=0.999)
    return model, tr


def test_training_reduces_loss(trained):
    model, tr = trained
    print(f"traces {len(tr.targets)}, loss {model.losses[0]:.3f} -> {model.losses[-1]:.3f}, "
          f"residual std {model.residual_std:.3f} decades")
    assert model.losses[-1] < 0.25 * model.losses[0]
    assert model.residual_std < 1.0


def test_learned_culling_gain_on_alkane(kx, trained):
    """Self-avoiding C40H82 against the paper's leaf-block method (Eq. 8 on
    leaf blocks, every shell quartet of a kept leaf block evaluated) at the
    same tau: the network drops leaf quartets and evaluates fewer shell
    quartets, and the K it gives stays within 1e-8 of that method's K.
    With the shell-level screen on, it never evaluates more."""
    import torch
    from paper_1401_6961_gb300 import learned
    model, _ = trained
    tau = 1e-8
    sys_ = wl.alkane(40, 6040, "small")
    P = torch.from_numpy(wl.density(sys_, 7040)).cuda()
    ex = kx.Exchange(sys_)
    K0 = ex(P, tau=tau, shell_screen=0).clone()
    base = ex.stats.n_shell_quartets
    K1, info = learned.learned_exchange(ex, P, model, tau, shell_screen=0)
    torch.cuda.synchronize()
    err = float((K1 - K0).abs().max())
    print(f"learned culling (margin {model.margin:.2f} decades): leaf quartets {info['leaf_quartets']} -> "
          f"{info['leaf_quartets_kept']} (bound <= 10 tau: {info['cullable']}), shell quartets {base} -> "
          f"{info['shell_quartets']}, max|dK| {err:.2e}")
    assert info["leaf_quartets_kept"] < info["leaf_quartets"]
    assert info["shell_quartets"] < base
    assert err <= 1e-8
    K2 = ex(P, tau=tau).clone()
    base2 = ex.stats.n_shell_quartets
    K3, info2 = learned.learned_exchange(ex, P, model, tau)
    err2 = float((K3 - K2).abs().max())
    print(f"with shell screen: shell quartets {base2} -> {info2['shell_quartets']}, max|dK| {err2:.2e}")
    assert info2["shell_quartets"] <= base2 and err2 <= 1e-8
    ex.close()


def test_learned_culling_against_oracle_rows(kx, trained):
    """Self-avoiding C14H30: the learned build's K rows of sampled shells
    against the oracle's leaf-block method at the same tau."""
    import torch
    import oracle
    from paper_1401_6961_gb300 import learned
    model, _ = trained
    tau = 1e-8
    sys_ = wl.alkane(14, 6014, "small")
    Pn = wl.density(sys_, 7014)
    ex = kx.Exchange(sys_)
    K1, info = learned.learned_exchange(ex, torch.from_numpy(Pn).cuda(), model, tau, shell_screen=0)
    rows = [int(x) for x in np.random.default_rng(14).choice(sys_.n_shell, 6, replace=False)]
    Kr, *_ = oracle.exchange_screened(sys_, Pn, tau, shell_screen=False, rows=rows)
    off = sys_.shell_offset
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows])
    assert np.abs(K1.cpu().numpy()[idx] - Kr[idx]).max() <= 1e-8
    assert info["leaf_quartets_kept"] <= info["leaf_quartets"]
    ex.close()


def test_learned_culling_is_safe_on_water256(kx, trained):
    """(H2O)256, small basis, tau = 1e-8: many cullable quartets per K block,
    the case where a root-sum-square budget broke the bar; the linear
    per-block budget keeps the learned build within 1e-8."""
    import torch
    from paper_1401_6961_gb300 import learned
    model, _ = trained
    tau = 1e-8
    sys_ = wl.water_sweep(256, "small")
    P = torch.from_numpy(wl.density(sys_, 5256)).cuda()
    ex = kx.Exchange(sys_)
    K0 = ex(P, tau=tau, precision=kx.KX_MIXED, split_threshold=5e-4).clone()
    base = ex.stats.n_shell_quartets
    K1, info = learned.learned_exchange(ex, P, model, tau, precision=kx.KX_MIXED, split_threshold=5e-4)
    err = float((K1 - K0).abs().max())
    print(f"(H2O)256: leaf quartets {info['leaf_quartets']} -> {info['leaf_quartets_kept']}, shell quartets "
          f"{base} -> {info['shell_quartets']}, max|dK| {err:.2e}")
    assert info["shell_quartets"] <= base and err <= 1e-8
    ex.close()


def test_learned_culling_in_symmetric_mixed_builds(kx, trained):
    """The learned build with the options of the benchmark's build
    (symmetric traversal, mixed precision, double words above the split):
    it traverses only K blocks with A <= C, mirrors the rest, and stays
    within 1e-8 of the plain FP64 build of every K block."""
    import torch
    from paper_1401_6961_gb300 import learned
    model, _ = trained
    tau = 1e-8
    sys_ = wl.water_cluster(16, 16, "small")
    P = torch.from_numpy(wl.density(sys_, 1016)).cuda()
    ex = kx.Exchange(sys_)
    K64 = ex(P, tau=tau).clone()
    full = ex.stats.n_leaf_quartets
    K1, info = learned.learned_exchange(ex, P, model, tau, symmetric=1, precision=kx.KX_MIXED_DW,
                                        split_threshold=5e-4)
    err = float((K1 - K64).abs().max())
    print(f"symmetric learned build: leaf quartets {info['leaf_quartets']} of {full}, kept "
          f"{info['leaf_quartets_kept']}, max|dK| {err:.2e}")
    assert info["leaf_quartets"] < 0.6 * full
    assert err <= 1e-8
    ex.close()


def test_cull_never_drops_quartets_above_ten_tau(kx, trained):
    import torch
    model, _ = trained
    sys_, Pn = wl.workload("water4")
    P = torch.from_numpy(Pn).cuda()
    ex = kx.Exchange(sys_)
    tau = 1e-8
    n = kx.kx_traverse(ex.ctx, P.data_ptr(), P.stride(0), kx.kx_default_opts(tau=tau))
    feat = torch.empty((n, 10), dtype=torch.float32, device="cuda")
    kx.kx_leaf_features(ex.ctx, feat.data_ptr(), n)
    before = kx.kx_get_worklist(ex.ctx, None, cap=n)
    lb = feat[:, 3].cpu().numpy()
    pred = torch.full((n,), -1e30, dtype=torch.float32, device="cuda")   # predicts "cull everything"
    kept = kx.kx_cull_kept(ex.ctx, pred.data_ptr(), tau, math.log10(0.5 * tau))
    after = kx.kx_get_worklist(ex.ctx, None, cap=max(kept, 1))[:kept]
    # exactly the quartets with bound > 10 tau survive, in their order
    must = before[lb > math.log10(10 * tau) + 1e-6]
    assert kept >= len(must)
    keep_set = {tuple(x) for x in after}
    assert all(tuple(x) in keep_set for x in must)
    ex.close()
