"""Learned culling of leaf quartets: training traces, GPU training, culled builds.

A small network (10 -> 64 -> 64 -> 64 -> 1, GELU) predicts, from ten
descriptors of a leaf quartet (A,B,C,D), log10 of the Frobenius norm of its
contribution to the K block (A,C).  The Schwarz x ||P|| bound of Eq. 8 is a
loose upper bound of that norm; quartets predicted far below it can be
skipped.  The exact bound stays the safety net: a quartet whose bound
exceeds 10 tau is always evaluated.

This module is the driver (argument marshalling and the training loop):
the traversal, the features, the targets, the forward/backward passes, the
optimiser steps, the BF16 inference, the cull and the ERI stage all run in
the library's CUDA kernels through the C ABI.

Traces: the kept leaf quartets of the plain traversal are sampled and
evaluated -- every shell quartet of the leaf block, i.e. with the shell-level
screen off, so that the target is the true contribution of the block -- in
batches whose (A,C) blocks are pairwise distinct, so that every quartet of a
batch owns its K block; the block norms are then the exact contribution
norms.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import _binding as B

NF, NH, NP = B.KX_NFEAT, B.KX_MLP_HIDDEN, B.KX_MLP_NPARAM
P_MU, P_IS, P_W1 = 0, NF, 2 * NF
P_B1 = P_W1 + NH * NF
P_W2 = P_B1 + NH
P_B2 = P_W2 + NH * NH
P_W3 = P_B2 + NH
P_B3 = P_W3 + NH * NH
P_W4 = P_B3 + NH
P_B4 = P_W4 + NH
LOG_FLOOR = -30.0   # log10 floor for contributions that vanish (by symmetry)


def _torch():
    import torch
    return torch


@dataclasses.dataclass
class Traces:
    features: np.ndarray      # (n, 10) float32
    targets: np.ndarray       # (n,) float32, log10 ||dK_AC||_F
    log10_beta: np.ndarray    # (n,) float32, the Eq. 8 bound of the quartet

    def __add__(self, o: "Traces") -> "Traces":
        return Traces(np.concatenate([self.features, o.features]), np.concatenate([self.targets, o.targets]),
                      np.concatenate([self.log10_beta, o.log10_beta]))


def traces(ex, P, tau: float, max_samples: int = 40000, seed: int = 0) -> Traces:
    """Samples of (features, exact log10 contribution) from the traversal of
    ``ex`` (an ``Exchange``) for the device density ``P`` at ``tau``."""
    torch = _torch()
    ctx = ex.ctx
    o = B.kx_default_opts(tau=tau)
    o_eval = B.kx_default_opts(tau=tau, shell_screen=0)
    n = B.kx_traverse(ctx, P.data_ptr(), P.stride(0), o)
    if n == 0:
        return Traces(np.zeros((0, NF), np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32))
    feat = torch.empty((n, NF), dtype=torch.float32, device=P.device)
    B.kx_leaf_features(ctx, feat.data_ptr(), n)
    work = B.kx_get_worklist(ctx, None, cap=n)          # kept order = feature order
    leaves, _ = ex.leaves()
    nl = leaves.shape[0]
    rng = np.random.default_rng(seed)
    key = work[:, 0].astype(np.int64) * nl + work[:, 2]
    groups = int(np.unique(key).shape[0])
    per_group = max(1, int(math.ceil(max_samples / groups)))
    # rank of every quartet inside its (A,C) group, in a random order
    order = rng.permutation(n)
    ks = key[order]
    srt = np.argsort(ks, kind="stable")
    ks_sorted = ks[srt]
    starts = np.r_[0, np.nonzero(np.diff(ks_sorted))[0] + 1]
    rank_sorted = np.arange(n) - np.repeat(starts, np.diff(np.r_[starts, n]))
    rank = np.empty(n, dtype=np.int64)
    rank[order[srt]] = rank_sorted
    sel = np.nonzero(rank < per_group)[0]
    tgt = np.full(n, np.nan, dtype=np.float64)
    K = torch.empty_like(P)
    for r in range(per_group):
        idx = sel[rank[sel] == r]
        if idx.shape[0] == 0:
            break
        B.kx_exchange_leaves(ctx, P.data_ptr(), P.stride(0), work[idx], o_eval, K.data_ptr(), K.stride(0))
        norms = B.kx_block_norms(ctx, K.data_ptr(), K.stride(0), work[idx])
        tgt[idx] = np.log10(np.maximum(norms, 10.0 ** LOG_FLOOR))
    f = feat[torch.from_numpy(sel).to(P.device)].cpu().numpy()
    return Traces(f, tgt[sel].astype(np.float32), f[:, 3].copy())


def init_params(tr: Traces, seed: int = 0) -> np.ndarray:
    """Normalisation from the trace features, Glorot-uniform weights, the
    output bias at the mean target."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NP, dtype=np.float32)
    mu = tr.features.mean(axis=0)
    sd = tr.features.std(axis=0)
    p[P_MU:P_MU + NF] = mu
    p[P_IS:P_IS + NF] = 1.0 / np.where(sd > 1e-6, sd, 1.0)

    def glorot(n_out, n_in):
        a = math.sqrt(6.0 / (n_in + n_out))
        return rng.uniform(-a, a, size=(n_out, n_in)).astype(np.float32)
    p[P_W1:P_B1] = glorot(NH, NF).ravel()
    p[P_W2:P_B2] = glorot(NH, NH).ravel()
    p[P_W3:P_B3] = glorot(NH, NH).ravel()
    p[P_W4:P_B4] = glorot(1, NH).ravel()
    p[P_B4] = float(tr.targets.mean()) if tr.targets.size else 0.0
    return p


@dataclasses.dataclass
class Model:
    params: np.ndarray        # (NP,) float32
    residual_std: float       # std of (prediction - target) on the training traces
    losses: List[float]
    # decades added to every prediction by the cull: the q-quantile of
    # (target - prediction) on traces of systems kept out of training
    # (calibrate); None = margin * residual_std
    margin: Optional[float] = None
    margin_q: Optional[float] = None


def train(tr: Traces, epochs: int = 400, lr: float = 3e-3, batch: int = 8192, seed: int = 0,
          device: int = 0) -> Model:
    """Adam on 0.5 * mean squared error of the log10 targets, with the
    library's forward/backward and update kernels."""
    torch = _torch()
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev).cuda_stream
    prm = torch.from_numpy(init_params(tr, seed)).to(dev)
    m = torch.zeros_like(prm)
    v = torch.zeros_like(prm)
    g = torch.zeros_like(prm)
    X = torch.from_numpy(np.ascontiguousarray(tr.features)).to(dev)
    Y = torch.from_numpy(np.ascontiguousarray(tr.targets)).to(dev)
    n = X.shape[0]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    step = 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen).to(dev)
        tot = 0.0
        for i0 in range(0, n, batch):
            idx = perm[i0:i0 + batch]
            xb = X[idx].contiguous()
            yb = Y[idx].contiguous()
            tot += B.kx_mlp_loss_grad(prm.data_ptr(), xb.data_ptr(), yb.data_ptr(), xb.shape[0], g.data_ptr(),
                                      stream) * xb.shape[0]
            step += 1
            B.kx_mlp_adam(prm.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), lr, step, stream)
        losses.append(tot / n)
    pred = predict(prm, X, device)
    res = (pred - Y).float()
    torch.cuda.synchronize(dev)
    return Model(prm.cpu().numpy(), float(res.std().item()), losses)


def calibrate(model: Model, held_out: Traces, q: float = 0.999, device: int = 0) -> Model:
    """The same network with its cull margin set from held-out traces: the
    q-quantile of how far the true log10 contribution lies above the BF16
    prediction, over systems of a family the network was not trained on (a
    distribution-free margin, unlike the Gaussian residual_std)."""
    torch = _torch()
    dev = torch.device("cuda", device)
    X = torch.from_numpy(np.ascontiguousarray(held_out.features)).to(dev)
    pred = predict(model.params, X, device).cpu().numpy().astype(np.float64)
    under = held_out.targets.astype(np.float64) - pred
    return dataclasses.replace(model, margin=max(0.0, float(np.quantile(under, q))), margin_q=q)


def predict(params, X, device: int = 0):
    """BF16 inference of the network on device features X (n, 10)."""
    torch = _torch()
    dev = torch.device("cuda", device)
    prm = params if isinstance(params, torch.Tensor) else torch.from_numpy(params).to(dev)
    out = torch.empty((X.shape[0],), dtype=torch.float32, device=dev)
    B.kx_mlp_infer_bf16(prm.data_ptr(), X.data_ptr(), X.shape[0], out.data_ptr(),
                        torch.cuda.current_stream(dev).cuda_stream)
    return out


def learned_exchange(ex, P, model: Model, tau: float, budget: Optional[float] = None, margin: float = 2.0,
                     K=None, **opts):
    """K with learned culling: traversal, features, BF16 inference, cull,
    then the ERI stage over what remains.  Returns (K, info).

    A leaf quartet of bound <= 10 tau is dropped when its predicted
    contribution, raised by the model's calibrated margin (else by
    ``margin`` residual standard deviations) and multiplied by the number of
    such quartets in its K block, is below ``budget`` (default tau / 10):
    the predicted sum of what any K block loses stays below the budget."""
    torch = _torch()
    ctx = ex.ctx
    o = B.kx_default_opts(tau=tau, **opts)
    n = B.kx_traverse(ctx, P.data_ptr(), P.stride(0), o)
    feat = torch.empty((max(n, 1), NF), dtype=torch.float32, device=P.device)
    if n:
        B.kx_leaf_features(ctx, feat.data_ptr(), n)
    pred = predict(model.params, feat[:n], ex.device) if n else feat[:0, 0]
    lb = math.log10(0.1 * tau if budget is None else budget)
    # the margin shifts every prediction up: pred + margin + log10(m) < log10(budget)
    shift = model.margin if model.margin is not None else margin * model.residual_std
    kept = B.kx_cull_kept(ctx, pred.data_ptr(), tau, lb - shift) if n else 0
    if K is None:
        K = torch.empty_like(P)
    st = B.kx_evaluate_kept(ctx, P.data_ptr(), P.stride(0), o, K.data_ptr(), K.stride(0))
    band = int((feat[:n, 3] <= math.log10(10.0 * tau)).sum().item()) if n else 0
    return K, {"leaf_quartets": n, "leaf_quartets_kept": kept, "cullable": band, "shell_quartets": st.n_shell_quartets,
               "flops": st.flops_fp64 + st.flops_fp32, "ms_total": st.ms_total}
