"""Plain FP64 CPU oracle for the screened exchange build -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package.  The library
itself never does.  The C source (``kxo.c``) shares nothing with the CUDA
library; see its header for the recurrences and the passages of the paper
each routine follows.

Parity status of each routine (what pins it, in ``tests/test_oracle_*.py``):

* ``boys``                 mpmath incomplete gamma, closed forms at T = 0 and
                           via erf, the downward-recursion identity.
* ``eri``                  (ss|ss) closed form; every class up to (dd|dd) by
                           analytic centre derivatives of that closed form;
                           8-fold symmetry; Cauchy-Schwarz.
* ``overlap``              closed-form s-s overlap, centre derivatives.
* ``exchange_direct``      K = K^T, linearity in P, permutation covariance,
                           block-diagonal K for far fragments.
* ``hilbert_*``            unit steps along the curve on a full 8^3 grid.
* ``tree_build``           brute-force check of the split rule.
* ``traverse``             equals brute-force leaf enumeration.
* ``exchange_worklist``    tau = 0 equals ``exchange_direct``; the culled
                           error obeys the rigorous bound of Eq. 8.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkxo.so")
_LOCK = threading.Lock()
_LIB = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


class _Basis(ctypes.Structure):
    _fields_ = [("n_shell", ctypes.c_int32), ("center", _f64p), ("l", _i32p), ("alpha", _f64p)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "kxo.c")
    hdr = os.path.join(_HERE, "kxo.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-D_DEFAULT_SOURCE", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            L.kxo_boys.argtypes = [ctypes.c_int, ctypes.c_double, _f64p]
            L.kxo_eri.argtypes = [_f64p, ctypes.c_double, ctypes.c_int] * 4 + [_f64p]
            L.kxo_overlap.argtypes = [_f64p, ctypes.c_double, ctypes.c_int] * 2 + [_f64p]
            L.kxo_exchange_direct.argtypes = [ctypes.POINTER(_Basis), _f64p, _f64p]
            L.kxo_schwarz_sq.argtypes = [ctypes.POINTER(_Basis), ctypes.c_double, _f64p]
            L.kxo_pblock_sq.argtypes = [ctypes.POINTER(_Basis), _f64p, _f64p]
            L.kxo_hilbert_keys.argtypes = [ctypes.c_int, _f64p, _i64p]
            L.kxo_key_of_cell.argtypes = [_i32p, ctypes.c_int, _i64p]
            L.kxo_shell_order.argtypes = [ctypes.c_int, _f64p, ctypes.c_int, _i32p, _i32p]
            L.kxo_tree_build.argtypes = [ctypes.c_int, _i32p, ctypes.c_int] + [_i32p] * 5
            L.kxo_tree_build.restype = ctypes.c_int
            L.kxo_traverse.argtypes = [ctypes.POINTER(_Basis), _f64p, _i32p, ctypes.c_int,
                                       _i32p, _i32p, _i32p, _i32p, _f64p, ctypes.c_double,
                                       _i32p, ctypes.c_int, _i32p, ctypes.c_int64]
            L.kxo_traverse.restype = ctypes.c_int64
            L.kxo_leaf_bruteforce.argtypes = [ctypes.POINTER(_Basis), _f64p, _i32p, ctypes.c_int,
                                              _i32p, _i32p, _i32p, _f64p, ctypes.c_double,
                                              _i32p, ctypes.c_int64, _f64p]
            L.kxo_leaf_bruteforce.restype = ctypes.c_int64
            L.kxo_exchange_worklist.argtypes = [ctypes.POINTER(_Basis), _f64p, _i32p, ctypes.c_int,
                                                _i32p, _i32p, _i32p, _f64p, ctypes.c_double,
                                                ctypes.c_int, _i32p, ctypes.c_int64, _i32p,
                                                ctypes.c_int, _f64p]
            L.kxo_exchange_worklist.restype = ctypes.c_int64
            L.kxo_num_threads.restype = ctypes.c_int
            _LIB = L
    return _LIB


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def num_threads() -> int:
    return int(lib().kxo_num_threads())


# ---------------------------------------------------------------------------
# integrals
# ---------------------------------------------------------------------------

def boys(mmax: int, T: float) -> np.ndarray:
    F = np.zeros(mmax + 1)
    lib().kxo_boys(int(mmax), float(T), _p(F, _f64p))
    return F


NCART = (1, 3, 6)


def eri(A, a, la, B, b, lb, C, c, lc, D, d, ld) -> np.ndarray:
    """Normalised shell-quartet block (ab|cd), shape (na, nb, nc, nd)."""
    cs = [np.ascontiguousarray(x, dtype=np.float64) for x in (A, B, C, D)]
    out = np.zeros(NCART[la] * NCART[lb] * NCART[lc] * NCART[ld])
    lib().kxo_eri(_p(cs[0], _f64p), float(a), int(la), _p(cs[1], _f64p), float(b), int(lb),
                  _p(cs[2], _f64p), float(c), int(lc), _p(cs[3], _f64p), float(d), int(ld),
                  _p(out, _f64p))
    return out.reshape(NCART[la], NCART[lb], NCART[lc], NCART[ld])


def overlap(A, a, la, B, b, lb) -> np.ndarray:
    cs = [np.ascontiguousarray(x, dtype=np.float64) for x in (A, B)]
    out = np.zeros(NCART[la] * NCART[lb])
    lib().kxo_overlap(_p(cs[0], _f64p), float(a), int(la), _p(cs[1], _f64p), float(b), int(lb),
                      _p(out, _f64p))
    return out.reshape(NCART[la], NCART[lb])


class Basis:
    """Keeps the arrays of a kxo_basis alive."""

    def __init__(self, sys_):
        self.center = np.ascontiguousarray(sys_.xyz[sys_.shell_atom], dtype=np.float64)
        self.l = np.ascontiguousarray(sys_.shell_l, dtype=np.int32)
        self.alpha = np.ascontiguousarray(sys_.shell_alpha, dtype=np.float64)
        self.n_shell = int(self.l.shape[0])
        self.s = _Basis(self.n_shell, _p(self.center, _f64p), _p(self.l, _i32p), _p(self.alpha, _f64p))
        self.n_fn = int(sum(NCART[x] for x in self.l))

    def ref(self):
        return ctypes.byref(self.s)


def exchange_direct(sys_, P: np.ndarray) -> np.ndarray:
    """K_{mu nu} = sum_{lam sig} (mu lam|nu sig) P_{lam sig}, every quartet."""
    b = Basis(sys_)
    P = np.ascontiguousarray(P, dtype=np.float64)
    K = np.zeros((b.n_fn, b.n_fn))
    lib().kxo_exchange_direct(b.ref(), _p(P, _f64p), _p(K, _f64p))
    return K


def schwarz_sq(sys_, tau_ovlp: float = 0.0) -> np.ndarray:
    b = Basis(sys_)
    s2 = np.zeros((b.n_shell, b.n_shell))
    lib().kxo_schwarz_sq(b.ref(), float(tau_ovlp), _p(s2, _f64p))
    return s2


def pblock_sq(sys_, P: np.ndarray) -> np.ndarray:
    b = Basis(sys_)
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.zeros((b.n_shell, b.n_shell))
    lib().kxo_pblock_sq(b.ref(), _p(P, _f64p), _p(out, _f64p))
    return out


# ---------------------------------------------------------------------------
# order, tree, traversal
# ---------------------------------------------------------------------------

def hilbert_keys(xyz: np.ndarray) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    k = np.zeros(xyz.shape[0], dtype=np.int64)
    lib().kxo_hilbert_keys(int(xyz.shape[0]), _p(xyz, _f64p), _p(k, _i64p))
    return k


def key_of_cell(q, bits: int) -> int:
    q = np.ascontiguousarray(q, dtype=np.int32)
    k = np.zeros(1, dtype=np.int64)
    lib().kxo_key_of_cell(_p(q, _i32p), int(bits), _p(k, _i64p))
    return int(k[0])


def shell_order(sys_) -> np.ndarray:
    xyz = np.ascontiguousarray(sys_.xyz, dtype=np.float64)
    sa = np.ascontiguousarray(sys_.shell_atom, dtype=np.int32)
    perm = np.zeros(sys_.n_shell, dtype=np.int32)
    lib().kxo_shell_order(int(xyz.shape[0]), _p(xyz, _f64p), int(sys_.n_shell), _p(sa, _i32p),
                          _p(perm, _i32p))
    return perm


class Tree:
    """Ragged bisection tree over tree-ordered shells (node 0 = root)."""

    def __init__(self, lo, hi, child0, child1, depth, perm):
        self.lo, self.hi, self.child0, self.child1, self.depth = lo, hi, child0, child1, depth
        self.perm = perm
        self.n_node = int(lo.shape[0])
        leaves = [v for v in range(self.n_node) if child0[v] < 0]
        leaves.sort(key=lambda v: lo[v])
        self.leaf_node = np.array(leaves, dtype=np.int32)

    @property
    def n_leaf(self) -> int:
        return int(self.leaf_node.shape[0])

    def leaf_ranges(self) -> np.ndarray:
        return np.stack([self.lo[self.leaf_node], self.hi[self.leaf_node]], axis=1)


def tree_build(sys_, leaf_max: int = 10, perm: Optional[np.ndarray] = None) -> Tree:
    if perm is None:
        perm = shell_order(sys_)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    nfn = np.ascontiguousarray(np.array([NCART[l] for l in sys_.shell_l[perm]], dtype=np.int32))
    n = sys_.n_shell
    arrs = [np.zeros(2 * n, dtype=np.int32) for _ in range(5)]
    nn = lib().kxo_tree_build(int(n), _p(nfn, _i32p), int(leaf_max), *[_p(a, _i32p) for a in arrs])
    lo, hi, c0, c1, dep = [a[:nn].copy() for a in arrs]
    return Tree(lo, hi, c0, c1, dep, perm)


def traverse(sys_, P: np.ndarray, tree: Tree, s2: np.ndarray, tau: float,
             rows: Optional[Sequence[int]] = None, cap: int = 1 << 22) -> np.ndarray:
    """Leaf quartets (A,B,C,D) kept by the depth-first traversal."""
    b = Basis(sys_)
    P = np.ascontiguousarray(P, dtype=np.float64)
    s2 = np.ascontiguousarray(s2, dtype=np.float64)
    rows_a = np.ascontiguousarray(np.asarray(rows if rows is not None else [], dtype=np.int32))
    while True:
        out = np.zeros((max(cap, 1), 4), dtype=np.int32)
        n = lib().kxo_traverse(b.ref(), _p(P, _f64p), _p(tree.perm, _i32p), tree.n_node,
                               _p(tree.lo, _i32p), _p(tree.hi, _i32p), _p(tree.child0, _i32p),
                               _p(tree.child1, _i32p), _p(s2, _f64p), float(tau),
                               _p(rows_a, _i32p), int(rows_a.shape[0]), _p(out, _i32p), int(cap))
        if n < 0:
            raise MemoryError("oracle traversal failed")
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def leaf_bruteforce(sys_, P: np.ndarray, tree: Tree, s2: np.ndarray, tau: float
                    ) -> Tuple[np.ndarray, np.ndarray]:
    b = Basis(sys_)
    P = np.ascontiguousarray(P, dtype=np.float64)
    s2 = np.ascontiguousarray(s2, dtype=np.float64)
    cap = tree.n_leaf ** 4
    out = np.zeros((max(cap, 1), 4), dtype=np.int32)
    beta = np.zeros(max(cap, 1))
    n = lib().kxo_leaf_bruteforce(b.ref(), _p(P, _f64p), _p(tree.perm, _i32p), tree.n_node,
                                  _p(tree.lo, _i32p), _p(tree.hi, _i32p), _p(tree.child0, _i32p),
                                  _p(s2, _f64p), float(tau), _p(out, _i32p), int(cap), _p(beta, _f64p))
    return out[:n].copy(), beta[:n].copy()


def exchange_worklist(sys_, P: np.ndarray, tree: Tree, s2: np.ndarray, tau: float,
                      work: np.ndarray, shell_screen: bool = True,
                      rows: Optional[Sequence[int]] = None) -> Tuple[np.ndarray, int]:
    """K over the leaf quartets of ``work`` (+ shell-level Eq. 8 screen)."""
    b = Basis(sys_)
    P = np.ascontiguousarray(P, dtype=np.float64)
    s2 = np.ascontiguousarray(s2, dtype=np.float64)
    work = np.ascontiguousarray(work, dtype=np.int32)
    rows_a = np.ascontiguousarray(np.asarray(rows if rows is not None else [], dtype=np.int32))
    K = np.zeros((b.n_fn, b.n_fn))
    n = lib().kxo_exchange_worklist(b.ref(), _p(P, _f64p), _p(tree.perm, _i32p), tree.n_node,
                                    _p(tree.lo, _i32p), _p(tree.hi, _i32p), _p(tree.child0, _i32p),
                                    _p(s2, _f64p), float(tau), int(bool(shell_screen)),
                                    _p(work, _i32p), int(work.shape[0]), _p(rows_a, _i32p),
                                    int(rows_a.shape[0]), _p(K, _f64p))
    return K, int(n)


def exchange_screened(sys_, P: np.ndarray, tau: float, leaf_max: int = 10,
                      shell_screen: bool = True, tau_ovlp: float = 0.0,
                      rows: Optional[Sequence[int]] = None):
    """The method end to end: order, tree, Schwarz, traversal, contraction.

    Returns (K, worklist, n_shell_quartets, tree, s2).
    """
    tree = tree_build(sys_, leaf_max)
    s2 = schwarz_sq(sys_, tau_ovlp)
    work = traverse(sys_, P, tree, s2, tau, rows=rows)
    K, nq = exchange_worklist(sys_, P, tree, s2, tau, work, shell_screen, rows=rows)
    return K, work, nq, tree, s2
