"""Occurrences of the permutational-symmetry cases of Eqs. 9-10 among the
leaf quartets a build keeps.

A kept leaf quartet (A,B,C,D) is the integral block (AB|CD) contracted with
P_BD into K_AC.  The same integrals serve up to eight ordered quartets: the
swaps inside the bra (BA|CD) and the ket (AB|DC), and bra with ket (CD|AB).
Eq. 10's canonical restriction keeps one representative of each set, and
Eq. 9 (EqA) applies all four K updates of a full set (the bra-ket swap is the
transpose of K, which a symmetric build already uses).  Per canonical
integral block this module counts how many distinct ordered images it has
(1, 2, 4 or 8: fewer when index blocks coincide) and how many of them the
traversal kept (each with its own P link in Eq. 8):

* "full": eight distinct images, all kept -- the 4-fold case of EqA;
* "coincident": fewer distinct images (A = B, C = D or (A,B) = (C,D)), all
  kept -- the cases with factors of two and transposes (EqB-EqH);
* "sparse": some images culled by their own P link -- fewer than 4 of the
  linked blocks take part.

Host analysis of a worklist (kx_get_worklist of a build with every K block,
symmetric = 0); nothing of the build itself runs here.
"""
from __future__ import annotations

import numpy as np


def _images(q):
    a, b, c, d = q
    out = set()
    for (w, x) in ((a, b), (b, a)):
        for (y, z) in ((c, d), (d, c)):
            out.add((w, x, y, z))
            out.add((y, z, w, x))
    return out


def occurrence_counts(work) -> dict:
    """Counts of canonical integral blocks per case, and the number of kept
    quartets per canonical block (the reuse a full symmetric scheme could
    draw on)."""
    w = np.asarray(work, dtype=np.int64).reshape(-1, 4)
    if len(w) == 0:
        return {"quartets": 0, "blocks": 0, "full": 0, "coincident": 0, "sparse": 0, "quartets_per_block": 0.0}
    lo1, hi1 = np.minimum(w[:, 0], w[:, 1]), np.maximum(w[:, 0], w[:, 1])
    lo2, hi2 = np.minimum(w[:, 2], w[:, 3]), np.maximum(w[:, 2], w[:, 3])
    # order the two pairs: (lo, hi) lexicographic
    swap = (lo1 > lo2) | ((lo1 == lo2) & (hi1 > hi2))
    p0 = np.where(swap, lo2, lo1)
    p1 = np.where(swap, hi2, hi1)
    p2 = np.where(swap, lo1, lo2)
    p3 = np.where(swap, hi1, hi2)
    n = int(w.max()) + 1
    key = ((p0 * n + p1) * n + p2) * n + p3
    uniq, kept = np.unique(key, return_counts=True)
    q3 = uniq % n
    q2 = (uniq // n) % n
    q1 = (uniq // (n * n)) % n
    q0 = uniq // (n * n * n)
    # distinct images of the canonical block
    bra_eq = q0 == q1
    ket_eq = q2 == q3
    pair_eq = (q0 == q2) & (q1 == q3)
    m = np.full(len(uniq), 8)
    m = np.where(bra_eq ^ ket_eq, 4, m)
    m = np.where(bra_eq & ket_eq, 2, m)
    m = np.where(pair_eq & ~(bra_eq | ket_eq), 4, m)
    m = np.where(pair_eq & bra_eq, 1, m)
    full = int(((m == 8) & (kept == m)).sum())
    coincident = int(((m < 8) & (kept == m)).sum())
    sparse = int((kept < m).sum())
    return {"quartets": int(len(w)), "blocks": int(len(uniq)), "full": full, "coincident": coincident,
            "sparse": sparse, "quartets_per_block": float(len(w)) / len(uniq)}


def integral_share(counts_by_class) -> float:
    """Share of the algorithmic FLOPs that does not involve P, for shell
    quartet counts per class (length 81), from the library's own counter."""
    from . import _binding as kb
    tot = integ = 0.0
    for cls, n in enumerate(counts_by_class):
        if n:
            t, i = kb.kx_class_flops(cls)
            tot += n * t
            integ += n * i
    return integ / tot if tot else 0.0
