"""The split threshold from an FP32 error budget (kx_split_plan,
kx_opts.split_budget).

The planner's 5-sigma estimate of max|dK| from the FP32 quartets must hold
for the build it chooses: the measured max|dK| of that mixed build against
the FP64 build of the same system (the same quartets, so only the FP32
rounding differs) stays at or below the estimate, and the estimate at or
below the budget.  The split grows with the budget; a budget below every
estimate gives split 0 (every quartet above the split); the budget option of
kx_exchange and of captured builds picks the planner's split.  The chosen
build also meets the mixed contract (1e-8) against the oracle.
"""
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


@pytest.mark.parametrize("name,tau,leaf", [("water16", 1e-10, 16), ("water16", 1e-8, 16), ("water4", 1e-10, 4)])
def test_estimate_holds_for_the_chosen_split(kx, name, tau, leaf):
    import torch
    sys_, P = wl.workload(name)
    ex = kx.Exchange(sys_, leaf_max=leaf)
    Pd = torch.from_numpy(P).cuda()
    budget = 5e-9
    sp = ex.split_plan(Pd, budget, tau=tau, symmetric=1)
    print(f"{name} tau {tau:g}: split {sp.split_used:.3g}, estimate {sp.fp32_err_estimate:.3g}, "
          f"bound {sp.fp32_err_bound:.3g}")
    assert sp.split_used > 0 and 0 < sp.fp32_err_estimate <= budget
    assert sp.fp32_err_bound >= sp.fp32_err_estimate / 5.0
    K64 = ex(Pd, tau=tau, symmetric=1).clone()
    Km = ex(Pd, tau=tau, symmetric=1, precision=kx.KX_MIXED, split_threshold=sp.split_used).clone()
    assert ex.stats.n_shell_quartets_fp64 < ex.stats.n_shell_quartets
    err = (Km - K64).abs().max().item()
    print(f"  measured max|dK| vs FP64 {err:.3g}")
    assert err <= sp.fp32_err_estimate
    # the budget option of kx_exchange builds with the planner's split
    Kb = ex(Pd, tau=tau, symmetric=1, precision=kx.KX_MIXED, split_budget=budget).clone()
    assert ex.stats.split_used == sp.split_used
    # (the planner's block sums are FP64 atomic adds, in no fixed order)
    assert ex.stats.fp32_err_estimate == pytest.approx(sp.fp32_err_estimate, rel=1e-12)
    # (the planning pass changes the leaf chunking, and so the FP32 warp sums)
    assert (Kb - Km).abs().max().item() <= 2 * sp.fp32_err_estimate
    if name == "water4":
        Kr, *_ = oracle.exchange_screened(sys_, P, tau, leaf_max=leaf)
        assert np.abs(Km.cpu().numpy() - Kr).max() <= 1e-8
    ex.close()


def test_split_grows_with_the_budget(kx):
    import torch
    sys_, P = wl.workload("water16")
    ex = kx.Exchange(sys_, leaf_max=16)
    Pd = torch.from_numpy(P).cuda()
    splits = [ex.split_plan(Pd, b, tau=1e-10, symmetric=1).split_used for b in (1e-10, 1e-9, 1e-8, 1e-7)]
    assert all(x <= y for x, y in zip(splits, splits[1:])) and splits[-1] > splits[0]
    sp = ex.split_plan(Pd, 1e-20, tau=1e-10, symmetric=1)
    assert sp.split_used == 0.0
    ex(Pd, tau=1e-10, symmetric=1, precision=kx.KX_MIXED, split_budget=1e-20)
    assert ex.stats.n_shell_quartets_fp64 == ex.stats.n_shell_quartets
    ex.close()


def test_captured_build_takes_the_planned_split(kx):
    import torch
    sys_, P = wl.workload("water16")
    ex = kx.Exchange(sys_, leaf_max=16)
    Pd = torch.from_numpy(P).cuda()
    opts = dict(tau=1e-10, symmetric=1, precision=kx.KX_MIXED)
    sp = ex.split_plan(Pd, 5e-9, **opts)
    K = torch.empty_like(Pd)
    ex.plan(Pd, K, split_budget=5e-9, **opts)
    assert ex.stats.split_used == sp.split_used
    ex.replay()
    torch.cuda.synchronize()
    assert ex.stats.split_used == sp.split_used
    assert ex.stats.fp32_err_estimate == pytest.approx(sp.fp32_err_estimate, rel=1e-12)
    Ke = ex(Pd, split_threshold=sp.split_used, **opts)
    assert (K - Ke).abs().max().item() <= 1e-8
    ex.close()


def test_budget_on_a_batch_is_not_implemented(kx):
    import torch
    systems, dens = wl.batch_workload(count=3)
    bx = kx.BatchExchange(systems)
    P = bx.pack([torch.from_numpy(d).cuda() for d in dens])
    with pytest.raises(kx.KxError) as e:
        bx(P, tau=1e-8, precision=kx.KX_MIXED, split_budget=5e-9)
    assert e.value.code == kx.KX_ENOTIMPL
    bx.close()
