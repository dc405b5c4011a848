"""Measures the per-class FP32 error constants of the split-precision model.

For every angular-momentum class (la,lb,lc,ld) it draws shell quartets of a
system (bounds beta spread over decades above 1e-9), evaluates each one in
FP32 and in FP64 through the library itself, and records
max|dK_block| / (eps32 beta) per quartet.  Single-shell leaves (leaf_max =
1) make every leaf quartet one shell quartet, and each batch of quartets has
pairwise distinct K blocks (a,c), so a K block holds exactly one quartet's
contribution.  Prints per class the number of quartets, the largest ratio,
its 99.9 % quantile and its root mean square, and the C tables of c_max
(1.5 x the largest ratio) and c_rms used by the split planner.

    python -m paper_1401_6961_gb300.calibrate [workload] [quartets_per_class]

Needs a GPU.  The workload is a name of ``workloads.workload`` (default
water16, the medium basis with d shells).
"""
from __future__ import annotations

import json
import sys

import numpy as np

EPS32 = 2.0 ** -24


def measure(name: str = "water16", per_class: int = 3000, seed: int = 7) -> dict:
    import torch

    import workloads as wl
    from . import _binding as kx

    kx.load()
    sys_, P = wl.workload(name)
    ex = kx.Exchange(sys_, device=0, leaf_max=1)
    Pd = torch.from_numpy(P).cuda()
    K = torch.empty_like(Pd)
    ex(Pd, out=K, tau=1e-14)          # P norms
    s2, pq = ex.norms()
    S, Pn = np.sqrt(s2), np.sqrt(pq)
    perm = ex.order()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    leaves, _ = ex.leaves()
    assert len(leaves) == len(perm) and (leaves[:, 0] == np.arange(len(perm))).all()
    n = sys_.n_fn
    L = np.asarray(sys_.shell_l)
    off, nf, ns = sys_.shell_offset, sys_.shell_nfn, sys_.n_shell
    rng = np.random.default_rng(seed)
    byl = [np.nonzero(L == l)[0] for l in range(3)]
    out = {}
    for cls in range(81):
        la, lb, lc, ld = cls // 27, (cls // 9) % 3, (cls // 3) % 3, cls % 3
        if min(len(byl[x]) for x in (la, lb, lc, ld)) == 0:
            continue
        m = 400000
        a, b, c, d = (rng.choice(byl[x], m) for x in (la, lb, lc, ld))
        beta = S[a, b] * Pn[b, d] * S[c, d]
        ok = beta > 1e-9
        a, b, c, d, beta = a[ok], b[ok], c[ok], d[ok], beta[ok]
        dec = np.floor(np.log10(beta)).astype(int)
        pick = np.concatenate([rng.permutation(np.nonzero(dec == x)[0])[: max(1, per_class // 12)]
                               for x in np.unique(dec)])
        a, b, c, d, beta = a[pick], b[pick], c[pick], d[pick], beta[pick]
        # rank of each quartet among those of its K block: batch = rank
        key = a * ns + c
        order = np.argsort(key, kind="stable")
        _, first, counts = np.unique(key[order], return_index=True, return_counts=True)
        rank = np.empty(len(key), int)
        rank[order] = np.arange(len(key)) - np.repeat(first, counts)
        ratio = []
        for bt in range(rank.max() + 1):
            sel = np.nonzero(rank == bt)[0]
            lv = np.stack([inv[a[sel]], inv[b[sel]], inv[c[sel]], inv[d[sel]]], 1).astype(np.int32)
            kx.kx_exchange_leaves(ex.ctx, Pd.data_ptr(), n, lv,
                                  kx.kx_default_opts(tau=0.0, precision=kx.KX_FP64, shell_screen=0),
                                  K.data_ptr(), n)
            K64 = K.cpu().numpy()
            kx.kx_exchange_leaves(ex.ctx, Pd.data_ptr(), n, lv,
                                  kx.kx_default_opts(tau=0.0, precision=kx.KX_MIXED, split_threshold=1e300,
                                                     shell_screen=0),
                                  K.data_ptr(), n)
            K32 = K.cpu().numpy()
            for q in sel:
                ra = slice(off[a[q]], off[a[q]] + nf[a[q]])
                rc = slice(off[c[q]], off[c[q]] + nf[c[q]])
                ratio.append(float(np.abs(K32[ra, rc] - K64[ra, rc]).max()) / (EPS32 * beta[q]))
        r = np.asarray(ratio)
        out[cls] = {"n": int(len(r)), "max": float(r.max()), "p999": float(np.quantile(r, 0.999)),
                    "rms": float(np.sqrt(np.mean(r * r)))}
    ex.close()
    return out


def tables(res: dict) -> str:
    """C initialisers of c_max and c_rms, nine classes per line."""
    cmax = [1.5 * res[c]["max"] if c in res else 10.0 for c in range(81)]
    crms = [res[c]["rms"] if c in res else 2.0 for c in range(81)]

    def lit(x):
        t = f"{x:.3g}"
        return (t if ("." in t or "e" in t) else t + ".0") + "f"

    def fmt(v):
        return "\n".join("    " + ", ".join(lit(x) for x in v[i:i + 9]) + "," for i in range(0, 81, 9))
    return "CMAX\n" + fmt(cmax) + "\nCRMS\n" + fmt(crms)


def main() -> None:
    name = sys.argv[1] if len(sys.argv) > 1 else "water16"
    per = int(sys.argv[2]) if len(sys.argv) > 2 else 3000
    res = measure(name, per)
    for c, v in sorted(res.items()):
        la, lb, lc, ld = c // 27, (c // 9) % 3, (c // 3) % 3, c % 3
        print(f"({'spd'[la]}{'spd'[lb]}|{'spd'[lc]}{'spd'[ld]}) {json.dumps(v)}")
    print(tables(res))


if __name__ == "__main__":
    main()
