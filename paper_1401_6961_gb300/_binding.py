"""ctypes binding of the C ABI in ``include/kx.h``.

Argument marshalling only: every function forwards to the entry point of
the same name in ``libkx.so``; all computation runs in the library's CUDA
kernels.  A missing library raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from .build import LIB

KX_OK, KX_EINVAL, KX_ESTATE, KX_ENOMEM, KX_ECUDA, KX_ECAPACITY, KX_ETIMEOUT, KX_ENOTIMPL = range(8)
KX_FP64, KX_MIXED, KX_MIXED_DW = 0, 1, 2
NSTREAM = 243   # class-kernel streams: precision (FP64, FP32, double word) * 81 + class
ERROR_NAMES = {0: "KX_OK", 1: "KX_EINVAL", 2: "KX_ESTATE", 3: "KX_ENOMEM", 4: "KX_ECUDA",
               5: "KX_ECAPACITY", 6: "KX_ETIMEOUT", 7: "KX_ENOTIMPL"}

# every entry point declared in include/kx.h
EXPORTS = ["kx_default_opts", "kx_create", "kx_build_schwarz", "kx_build_tree", "kx_exchange",
           "kx_exchange_host", "kx_count", "kx_create_batch", "kx_exchange_batch", "kx_exchange_batch_host",
           "kx_packed_size", "kx_autotune", "kx_get_launch_shapes", "kx_set_launch_shape", "kx_graph_plan", "kx_graph_launch",
           "kx_n_functions", "kx_get_order", "kx_get_leaves", "kx_get_worklist",
           "kx_get_norms", "kx_get_profile", "kx_peak_probe", "kx_traverse_level_noalloc",
           "kx_traverse", "kx_leaf_features", "kx_cull_kept", "kx_evaluate_kept", "kx_exchange_leaves",
           "kx_block_norms", "kx_mlp_infer_bf16", "kx_mlp_loss_grad", "kx_mlp_adam",
           "kx_row_work", "kx_shard_bounds", "kx_split_plan", "kx_class_flops", "kx_last_error", "kx_destroy"]
KX_NFEAT = 10
KX_MLP_HIDDEN = 64
KX_MLP_NPARAM = 9109
KX_NOALLOC_MAX_TASKS = 1 << 18
KX_PROBE_FP64_MMA = 2
KX_PROBE_DW = 3

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


class kx_basis(ctypes.Structure):
    _fields_ = [("n_atom", ctypes.c_int32), ("n_shell", ctypes.c_int32), ("xyz", _f64p),
                ("shell_atom", _i32p), ("shell_l", _i32p), ("shell_alpha", _f64p)]


class kx_opts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("split_threshold", ctypes.c_double),
                ("precision", ctypes.c_int32), ("shell_screen", ctypes.c_int32),
                ("keep_worklist", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("chunk_records", ctypes.c_int64), ("symmetric", ctypes.c_int32),
                ("row_leaf_lo", ctypes.c_int32), ("row_leaf_hi", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("split_budget", ctypes.c_double)]


class kx_stats(ctypes.Structure):
    _fields_ = [("n_leaf_quartets", ctypes.c_int64), ("n_shell_quartets", ctypes.c_int64),
                ("n_shell_quartets_fp64", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("n_shell_quartets_dw", ctypes.c_int64),
                ("n_tasks", ctypes.c_int64 * 32), ("depth", ctypes.c_int32), ("n_chunks", ctypes.c_int32),
                ("n_launches", ctypes.c_int32), ("pad", ctypes.c_int32), ("flops_fp64", ctypes.c_double),
                ("flops_fp32", ctypes.c_double), ("flops_dw", ctypes.c_double), ("ms_norms", ctypes.c_double),
                ("ms_traverse", ctypes.c_double), ("ms_expand", ctypes.c_double),
                ("ms_eri", ctypes.c_double), ("ms_eri_kernel_max", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("split_used", ctypes.c_double),
                ("fp32_err_bound", ctypes.c_double), ("fp32_err_estimate", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "n_tasks")}
        d["n_tasks"] = list(self.n_tasks)[: self.depth + 1]
        return d


class KxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return LIB


def load() -> ctypes.CDLL:
    """Loads libkx.so; raises ImportError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"{LIB} is not built; run paper_1401_6961_gb300.build.build() "
                          "(the CUDA library is required, there is no CPU path)")
    L = ctypes.CDLL(LIB)
    vp = ctypes.c_void_p
    L.kx_default_opts.argtypes = [ctypes.POINTER(kx_opts)]
    L.kx_default_opts.restype = None
    L.kx_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(kx_basis), ctypes.c_int, vp]
    L.kx_build_schwarz.argtypes = [vp, ctypes.c_double]
    L.kx_build_tree.argtypes = [vp, ctypes.c_int32, _i32p]
    L.kx_exchange.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(kx_opts), vp, ctypes.c_int64,
                              ctypes.POINTER(kx_stats)]
    L.kx_exchange_host.argtypes = [vp, _f64p, ctypes.c_int64, ctypes.POINTER(kx_opts), _f64p,
                                   ctypes.c_int64, ctypes.POINTER(kx_stats)]
    L.kx_count.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(kx_opts), ctypes.POINTER(kx_stats)]
    L.kx_create_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.POINTER(kx_basis), ctypes.c_int, vp]
    L.kx_exchange_batch.argtypes = [vp, vp, ctypes.POINTER(kx_opts), vp, ctypes.POINTER(kx_stats)]
    L.kx_exchange_batch_host.argtypes = [vp, _f64p, ctypes.POINTER(kx_opts), _f64p, ctypes.POINTER(kx_stats)]
    L.kx_autotune.argtypes = [vp, vp, ctypes.POINTER(kx_opts), vp, ctypes.POINTER(kx_stats), _i32p]
    L.kx_get_launch_shapes.argtypes = [vp, _i32p, _i32p, _i32p]
    L.kx_set_launch_shape.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.kx_graph_plan.argtypes = [vp, vp, ctypes.POINTER(kx_opts), vp, ctypes.c_double, ctypes.POINTER(kx_stats)]
    L.kx_graph_launch.argtypes = [vp, ctypes.POINTER(kx_stats)]
    L.kx_packed_size.argtypes = [vp]
    L.kx_packed_size.restype = ctypes.c_int64
    L.kx_n_functions.argtypes = [vp]
    L.kx_n_functions.restype = ctypes.c_int64
    L.kx_get_order.argtypes = [vp, _i32p]
    L.kx_get_leaves.argtypes = [vp, _i32p, _i32p, ctypes.c_int32, _i32p, _i32p]
    L.kx_get_worklist.argtypes = [vp, _i32p, ctypes.c_int32, _i32p, ctypes.c_int64, _i64p]
    L.kx_get_norms.argtypes = [vp, _f64p, _f64p]
    L.kx_get_profile.argtypes = [vp, _f64p, _i64p, _f64p, _i32p]
    L.kx_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, _f64p]
    L.kx_row_work.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(kx_opts), _f64p]
    L.kx_split_plan.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(kx_opts), ctypes.c_double,
                                ctypes.POINTER(kx_stats)]
    L.kx_shard_bounds.argtypes = [_f64p, ctypes.c_int32, ctypes.c_int32, _i32p]
    L.kx_class_flops.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.kx_traverse_level_noalloc.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_int64, ctypes.c_double, vp,
                                            ctypes.c_int64, _i64p]
    L.kx_traverse.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(kx_opts), _i64p]
    L.kx_leaf_features.argtypes = [vp, vp, ctypes.c_int64, _i64p]
    L.kx_cull_kept.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, _i64p]
    L.kx_evaluate_kept.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(kx_opts), vp, ctypes.c_int64,
                                   ctypes.POINTER(kx_stats)]
    L.kx_exchange_leaves.argtypes = [vp, vp, ctypes.c_int64, _i32p, ctypes.c_int64, ctypes.POINTER(kx_opts), vp,
                                     ctypes.c_int64, ctypes.POINTER(kx_stats)]
    L.kx_block_norms.argtypes = [vp, vp, ctypes.c_int64, _i32p, ctypes.c_int64, _f64p]
    L.kx_mlp_infer_bf16.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    L.kx_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int64, vp, _f64p, vp]
    L.kx_mlp_adam.argtypes = [vp, vp, vp, vp, ctypes.c_float, ctypes.c_int32, vp]
    L.kx_last_error.argtypes = [vp]
    L.kx_last_error.restype = ctypes.c_char_p
    L.kx_destroy.argtypes = [vp]
    L.kx_destroy.restype = None
    for name in EXPORTS:
        if name not in ("kx_default_opts", "kx_n_functions", "kx_packed_size", "kx_last_error", "kx_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _check(ctx, r: int):
    if r != KX_OK:
        msg = load().kx_last_error(ctx).decode() if ctx else "(no context)"
        raise KxError(r, msg)


# ---------------------------------------------------------------------------
# the C ABI, one wrapper per entry point
# ---------------------------------------------------------------------------

def kx_default_opts(**overrides) -> kx_opts:
    o = kx_opts()
    load().kx_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class _BasisArrays:
    def __init__(self, xyz, shell_atom, shell_l, shell_alpha):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.sa = np.ascontiguousarray(shell_atom, dtype=np.int32)
        self.sl = np.ascontiguousarray(shell_l, dtype=np.int32)
        self.al = np.ascontiguousarray(shell_alpha, dtype=np.float64)
        self.s = kx_basis(self.xyz.shape[0], self.sl.shape[0], _p(self.xyz, _f64p), _p(self.sa, _i32p),
                          _p(self.sl, _i32p), _p(self.al, _f64p))


def kx_create(xyz, shell_atom, shell_l, shell_alpha, device: int = 0, stream: int = 0) -> ctypes.c_void_p:
    """Context for a basis (bohr, bohr^-2); ``stream`` is a cudaStream_t handle."""
    b = _BasisArrays(xyz, shell_atom, shell_l, shell_alpha)
    ctx = ctypes.c_void_p()
    r = load().kx_create(ctypes.byref(ctx), ctypes.byref(b.s), int(device), ctypes.c_void_p(int(stream)))
    if r != KX_OK:
        raise KxError(r, "kx_create failed")
    return ctx


def kx_create_batch(systems, device: int = 0, stream: int = 0) -> ctypes.c_void_p:
    """Context for a batch of systems (each with xyz, shell_atom, shell_l, shell_alpha)."""
    arrs = [_BasisArrays(s.xyz, s.shell_atom, s.shell_l, s.shell_alpha) for s in systems]
    bases = (kx_basis * len(arrs))(*[a.s for a in arrs])
    ctx = ctypes.c_void_p()
    r = load().kx_create_batch(ctypes.byref(ctx), len(arrs), bases, int(device), ctypes.c_void_p(int(stream)))
    if r != KX_OK:
        raise KxError(r, "kx_create_batch failed")
    return ctx


def kx_exchange_batch(ctx, P_ptr: int, opts: kx_opts, K_ptr: int) -> kx_stats:
    """Device pointers (ints) to packed FP64 P and K (kx_packed_size doubles)."""
    st = kx_stats()
    _check(ctx, load().kx_exchange_batch(ctx, ctypes.c_void_p(P_ptr), ctypes.byref(opts), ctypes.c_void_p(K_ptr),
                                         ctypes.byref(st)))
    return st


def kx_exchange_batch_host(ctx, P: np.ndarray, opts: kx_opts, K: np.ndarray) -> kx_stats:
    assert P.dtype == np.float64 and K.dtype == np.float64 and P.flags["C_CONTIGUOUS"] and K.flags["C_CONTIGUOUS"]
    st = kx_stats()
    _check(ctx, load().kx_exchange_batch_host(ctx, P.ctypes.data_as(_f64p), ctypes.byref(opts),
                                              K.ctypes.data_as(_f64p), ctypes.byref(st)))
    return st


def kx_packed_size(ctx) -> int:
    return int(load().kx_packed_size(ctx))


def kx_autotune(ctx, P_ptr: int, opts: kx_opts, K_ptr: int) -> Tuple[kx_stats, int]:
    st = kx_stats()
    n = ctypes.c_int32()
    _check(ctx, load().kx_autotune(ctx, ctypes.c_void_p(P_ptr), ctypes.byref(opts), ctypes.c_void_p(K_ptr),
                                   ctypes.byref(st), ctypes.byref(n)))
    return st, int(n.value)


def kx_get_launch_shapes(ctx) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(threads, blocks per SM, kernel variant) of the NSTREAM streams."""
    t = np.zeros(NSTREAM, dtype=np.int32)
    b = np.zeros(NSTREAM, dtype=np.int32)
    v = np.zeros(NSTREAM, dtype=np.int32)
    _check(ctx, load().kx_get_launch_shapes(ctx, _p(t, _i32p), _p(b, _i32p), _p(v, _i32p)))
    return t, b, v


def kx_set_launch_shape(ctx, stream: int, threads: int, blocks_per_sm: int = 0, variant: int = 0) -> None:
    _check(ctx, load().kx_set_launch_shape(ctx, int(stream), int(threads), int(blocks_per_sm), int(variant)))


def kx_graph_plan(ctx, P_ptr: int, opts: kx_opts, K_ptr: int, headroom: float = 0.25) -> kx_stats:
    st = kx_stats()
    _check(ctx, load().kx_graph_plan(ctx, ctypes.c_void_p(P_ptr), ctypes.byref(opts), ctypes.c_void_p(K_ptr),
                                     float(headroom), ctypes.byref(st)))
    return st


def kx_graph_launch(ctx) -> kx_stats:
    st = kx_stats()
    _check(ctx, load().kx_graph_launch(ctx, ctypes.byref(st)))
    return st


def kx_build_schwarz(ctx, tau_ovlp: float = 0.0) -> None:
    _check(ctx, load().kx_build_schwarz(ctx, float(tau_ovlp)))


def kx_build_tree(ctx, leaf_max_functions: int = 10, perm: Optional[Sequence[int]] = None) -> None:
    if perm is None:
        _check(ctx, load().kx_build_tree(ctx, int(leaf_max_functions), None))
    else:
        pa = np.ascontiguousarray(perm, dtype=np.int32)
        _check(ctx, load().kx_build_tree(ctx, int(leaf_max_functions), _p(pa, _i32p)))


def kx_exchange(ctx, P_ptr: int, ldp: int, opts: kx_opts, K_ptr: int, ldk: int) -> kx_stats:
    """Device pointers (ints) to row-major FP64 P and K."""
    st = kx_stats()
    _check(ctx, load().kx_exchange(ctx, ctypes.c_void_p(P_ptr), int(ldp), ctypes.byref(opts),
                                   ctypes.c_void_p(K_ptr), int(ldk), ctypes.byref(st)))
    return st


def kx_exchange_host(ctx, P: np.ndarray, opts: kx_opts, K: np.ndarray) -> kx_stats:
    """Host arrays; P and K are row-major float64 (n_fn x n_fn, any ld)."""
    assert P.dtype == np.float64 and K.dtype == np.float64
    assert P.flags["C_CONTIGUOUS"] or P.strides[1] == 8
    st = kx_stats()
    _check(ctx, load().kx_exchange_host(ctx, P.ctypes.data_as(_f64p), P.strides[0] // 8, ctypes.byref(opts),
                                        K.ctypes.data_as(_f64p), K.strides[0] // 8, ctypes.byref(st)))
    return st


def kx_count(ctx, P_ptr: int, ldp: int, opts: kx_opts) -> kx_stats:
    """Survivor counts of a build (device P; ldp = 0 for a batch's packed P)."""
    st = kx_stats()
    _check(ctx, load().kx_count(ctx, ctypes.c_void_p(P_ptr), int(ldp), ctypes.byref(opts), ctypes.byref(st)))
    return st


def kx_n_functions(ctx) -> int:
    return int(load().kx_n_functions(ctx))


def kx_get_order(ctx, n_shell: int) -> np.ndarray:
    out = np.zeros(n_shell, dtype=np.int32)
    _check(ctx, load().kx_get_order(ctx, _p(out, _i32p)))
    return out


def kx_get_leaves(ctx) -> Tuple[np.ndarray, int]:
    """(leaves [n_leaf, 2] of [lo, hi) tree positions, depth)."""
    nl, dep = ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, load().kx_get_leaves(ctx, None, None, 0, ctypes.byref(nl), ctypes.byref(dep)))
    lo = np.zeros(nl.value, dtype=np.int32)
    hi = np.zeros(nl.value, dtype=np.int32)
    _check(ctx, load().kx_get_leaves(ctx, _p(lo, _i32p), _p(hi, _i32p), nl.value, ctypes.byref(nl),
                                     ctypes.byref(dep)))
    return np.stack([lo, hi], axis=1), int(dep.value)


def kx_get_worklist(ctx, a_filter: Optional[Sequence[int]] = None, cap: int = 1 << 22) -> np.ndarray:
    L = load()
    fa = np.ascontiguousarray(a_filter if a_filter is not None else [], dtype=np.int32)
    n = ctypes.c_int64()
    while True:
        out = np.zeros((max(cap, 1), 4), dtype=np.int32)
        r = L.kx_get_worklist(ctx, _p(fa, _i32p), int(fa.shape[0]), _p(out, _i32p), int(cap), ctypes.byref(n))
        if r == KX_ECAPACITY:
            cap = int(n.value)
            continue
        _check(ctx, r)
        return out[: n.value].copy()


def kx_get_norms(ctx, n_shell: int, with_p: bool = True, total: Optional[int] = None):
    """Dense [n_shell, n_shell] tables; for a batch pass ``total`` (sum of
    n_shell_y^2) to get the flat per-system blocks."""
    shape = (n_shell, n_shell) if total is None else (int(total),)
    s2 = np.zeros(shape)
    pq = np.zeros(shape) if with_p else None
    _check(ctx, load().kx_get_norms(ctx, _p(s2, _f64p), _p(pq, _f64p) if with_p else None))
    return s2, pq


def kx_get_profile(ctx) -> dict:
    """Per-stream totals of the last profiled build: arrays of NSTREAM entries
    indexed by precision * 81 + class (precision 0 = FP64)."""
    ms = np.zeros(NSTREAM)
    n = np.zeros(NSTREAM, dtype=np.int64)
    fl = np.zeros(NSTREAM)
    la = np.zeros(NSTREAM, dtype=np.int32)
    _check(ctx, load().kx_get_profile(ctx, _p(ms, _f64p), _p(n, _i64p), _p(fl, _f64p), _p(la, _i32p)))
    return {"ms": ms, "n": n, "flops": fl, "launches": la}


def kx_peak_probe(device: int = 0, precision: int = KX_FP64) -> float:
    """Measured throughput in GFLOP/s: the FMA pipe (FP64 or, with KX_MIXED,
    FP32), with KX_PROBE_FP64_MMA the FP64 tensor cores (DMMA), with
    KX_PROBE_DW double-word FP32 multiply-adds."""
    g = ctypes.c_double()
    r = load().kx_peak_probe(int(device), int(precision), ctypes.byref(g))
    if r != KX_OK:
        raise KxError(r, "kx_peak_probe failed")
    return float(g.value)


def kx_row_work(ctx, P_ptr: int, ldp: int, opts: kx_opts) -> np.ndarray:
    """Algorithmic FLOPs of the ERI stage per row leaf A (leaf ordinal) of
    the build with these options, from its traversal and count pass."""
    _, n_leaf = _n_leaves(ctx)
    w = np.zeros(n_leaf)
    _check(ctx, load().kx_row_work(ctx, ctypes.c_void_p(P_ptr), int(ldp), ctypes.byref(opts), _p(w, _f64p)))
    return w


def kx_split_plan(ctx, P_ptr: int, ldp: int, opts: kx_opts, budget: float) -> kx_stats:
    """Split threshold from the FP32 error model (split_used,
    fp32_err_estimate, fp32_err_bound of the returned stats)."""
    st = kx_stats()
    _check(ctx, load().kx_split_plan(ctx, ctypes.c_void_p(P_ptr), int(ldp), ctypes.byref(opts), float(budget),
                                     ctypes.byref(st)))
    return st


def kx_class_flops(cls: int):
    """(total, integral) algorithmic FLOPs of one quartet of class cls
    (host computation)."""
    t, i = ctypes.c_double(), ctypes.c_double()
    r = load().kx_class_flops(int(cls), ctypes.byref(t), ctypes.byref(i))
    if r != KX_OK:
        raise KxError(r, "kx_class_flops failed")
    return float(t.value), float(i.value)


def _n_leaves(ctx):
    nl, dep = ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, load().kx_get_leaves(ctx, None, None, 0, ctypes.byref(nl), ctypes.byref(dep)))
    return int(dep.value), int(nl.value)


def kx_shard_bounds(work, n_shards: int) -> np.ndarray:
    """Leaf boundaries [n_shards + 1] of contiguous row-block shards of
    balanced work (host computation, no device)."""
    w = np.ascontiguousarray(work, dtype=np.float64)
    b = np.zeros(int(n_shards) + 1, dtype=np.int32)
    r = load().kx_shard_bounds(_p(w, _f64p), int(w.shape[0]), int(n_shards), _p(b, _i32p))
    if r != KX_OK:
        raise KxError(r, "kx_shard_bounds failed")
    return b


def kx_traverse_level_noalloc(ctx, level: int, front_ptr: int, n: int, tau: float, next_ptr: int,
                              cap: int) -> int:
    """One traversal level without allocation; device pointers to uint16
    task arrays ([n][4] in, [cap][4] out).  Returns the next frontier size."""
    nn = ctypes.c_int64()
    _check(ctx, load().kx_traverse_level_noalloc(ctx, int(level), ctypes.c_void_p(front_ptr), int(n), float(tau),
                                                 ctypes.c_void_p(next_ptr), int(cap), ctypes.byref(nn)))
    return int(nn.value)


# --- learned culling ------------------------------------------------------

def kx_traverse(ctx, P_ptr: int, ldp: int, opts: kx_opts) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().kx_traverse(ctx, ctypes.c_void_p(P_ptr), int(ldp), ctypes.byref(opts), ctypes.byref(n)))
    return int(n.value)


def kx_leaf_features(ctx, feat_ptr: int, cap: int) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().kx_leaf_features(ctx, ctypes.c_void_p(feat_ptr), int(cap), ctypes.byref(n)))
    return int(n.value)


def kx_cull_kept(ctx, pred_ptr: int, tau: float, log10_budget: float) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().kx_cull_kept(ctx, ctypes.c_void_p(pred_ptr), float(tau), float(log10_budget),
                                    ctypes.byref(n)))
    return int(n.value)


def kx_evaluate_kept(ctx, P_ptr: int, ldp: int, opts: kx_opts, K_ptr: int, ldk: int) -> kx_stats:
    st = kx_stats()
    _check(ctx, load().kx_evaluate_kept(ctx, ctypes.c_void_p(P_ptr), int(ldp), ctypes.byref(opts),
                                        ctypes.c_void_p(K_ptr), int(ldk), ctypes.byref(st)))
    return st


def kx_exchange_leaves(ctx, P_ptr: int, ldp: int, leaves: np.ndarray, opts: kx_opts, K_ptr: int,
                       ldk: int) -> kx_stats:
    lv = np.ascontiguousarray(leaves, dtype=np.int32).reshape(-1, 4)
    st = kx_stats()
    _check(ctx, load().kx_exchange_leaves(ctx, ctypes.c_void_p(P_ptr), int(ldp), _p(lv, _i32p), int(lv.shape[0]),
                                          ctypes.byref(opts), ctypes.c_void_p(K_ptr), int(ldk), ctypes.byref(st)))
    return st


def kx_block_norms(ctx, K_ptr: int, ldk: int, leaves: np.ndarray) -> np.ndarray:
    lv = np.ascontiguousarray(leaves, dtype=np.int32).reshape(-1, 4)
    out = np.zeros(lv.shape[0])
    _check(ctx, load().kx_block_norms(ctx, ctypes.c_void_p(K_ptr), int(ldk), _p(lv, _i32p), int(lv.shape[0]),
                                      _p(out, _f64p)))
    return out


def _rc(r: int, what: str):
    if r != KX_OK:
        raise KxError(r, what)


def kx_mlp_infer_bf16(params_ptr: int, feat_ptr: int, n: int, pred_ptr: int, stream: int = 0) -> None:
    _rc(load().kx_mlp_infer_bf16(ctypes.c_void_p(params_ptr), ctypes.c_void_p(feat_ptr), int(n),
                                 ctypes.c_void_p(pred_ptr), ctypes.c_void_p(int(stream))), "kx_mlp_infer_bf16")


def kx_mlp_loss_grad(params_ptr: int, feat_ptr: int, target_ptr: int, n: int, grad_ptr: int,
                     stream: int = 0) -> float:
    loss = ctypes.c_double()
    _rc(load().kx_mlp_loss_grad(ctypes.c_void_p(params_ptr), ctypes.c_void_p(feat_ptr), ctypes.c_void_p(target_ptr),
                                int(n), ctypes.c_void_p(grad_ptr), ctypes.byref(loss), ctypes.c_void_p(int(stream))),
        "kx_mlp_loss_grad")
    return float(loss.value)


def kx_mlp_adam(params_ptr: int, grad_ptr: int, m_ptr: int, v_ptr: int, lr: float, step: int,
                stream: int = 0) -> None:
    _rc(load().kx_mlp_adam(ctypes.c_void_p(params_ptr), ctypes.c_void_p(grad_ptr), ctypes.c_void_p(m_ptr),
                           ctypes.c_void_p(v_ptr), float(lr), int(step), ctypes.c_void_p(int(stream))), "kx_mlp_adam")


def kx_last_error(ctx) -> str:
    return load().kx_last_error(ctx).decode()


def kx_destroy(ctx) -> None:
    if ctx:
        load().kx_destroy(ctx)


# ---------------------------------------------------------------------------
# convenience object over torch tensors
# ---------------------------------------------------------------------------

class Exchange:
    """A context for one molecule: ``Exchange(system)(P) -> K`` on the GPU.

    ``system`` has ``xyz`` (bohr), ``shell_atom``, ``shell_l`` and
    ``shell_alpha`` (bohr^-2), e.g. a ``workloads.System``.
    """

    def __init__(self, system, device: int = 0, leaf_max: int = 10, tau_ovlp: float = 0.0,
                 perm=None, stream=None):
        import torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.n_shell = int(len(system.shell_l))
        self.ctx = kx_create(system.xyz, system.shell_atom, system.shell_l, system.shell_alpha,
                             device, self.stream.cuda_stream)
        self.n_fn = kx_n_functions(self.ctx)
        kx_build_schwarz(self.ctx, tau_ovlp)
        kx_build_tree(self.ctx, leaf_max, perm)

    def __call__(self, P, out=None, **opts):
        import torch
        assert P.is_cuda and P.dtype == torch.float64 and P.stride(1) == 1
        n = self.n_fn
        assert P.shape == (n, n)
        K = out if out is not None else torch.empty((n, n), dtype=torch.float64, device=P.device)
        o = kx_default_opts(**opts)
        self.stats = kx_exchange(self.ctx, P.data_ptr(), P.stride(0), o, K.data_ptr(), K.stride(0))
        return K

    def host(self, P: np.ndarray, **opts) -> np.ndarray:
        K = np.zeros_like(P)
        self.stats = kx_exchange_host(self.ctx, np.ascontiguousarray(P), kx_default_opts(**opts), K)
        return K

    def count(self, P, **opts) -> kx_stats:
        """Survivor counts of the build ``self(P, **opts)`` without building K."""
        import torch
        assert P.is_cuda and P.dtype == torch.float64 and P.stride(1) == 1 and P.shape == (self.n_fn, self.n_fn)
        return kx_count(self.ctx, P.data_ptr(), P.stride(0), kx_default_opts(**opts))

    def autotune(self, P, out=None, **opts):
        """One build (P, K dense and contiguous) that also tunes the class
        kernels' launch shapes for later builds."""
        import torch
        assert P.is_contiguous() and P.shape == (self.n_fn, self.n_fn)
        K = out if out is not None else torch.empty_like(P)
        self.stats, self.n_tuned = kx_autotune(self.ctx, P.data_ptr(), kx_default_opts(**opts), K.data_ptr())
        return K

    def plan(self, P, K, headroom: float = 0.25, **opts):
        """Captures a build reading P and writing K (dense, contiguous, static
        buffers) into a CUDA graph; ``replay()`` rebuilds K from P's current
        contents."""
        assert P.is_contiguous() and K.is_contiguous() and P.shape == (self.n_fn, self.n_fn) == K.shape
        self.stats = kx_graph_plan(self.ctx, P.data_ptr(), kx_default_opts(**opts), K.data_ptr(), headroom)
        self._graph_bufs = (P, K)
        return K

    def replay(self):
        self.stats = kx_graph_launch(self.ctx)
        return self._graph_bufs[1]

    def row_work(self, P, **opts) -> np.ndarray:
        """Work (algorithmic FLOPs) per row leaf of the build ``self(P, **opts)``."""
        import torch
        assert P.is_cuda and P.dtype == torch.float64 and P.stride(1) == 1 and P.shape == (self.n_fn, self.n_fn)
        return kx_row_work(self.ctx, P.data_ptr(), P.stride(0), kx_default_opts(**opts))

    def split_plan(self, P, budget: float, **opts) -> kx_stats:
        """The split of a mixed build of P whose FP32 error estimate fits `budget`."""
        import torch
        assert P.is_cuda and P.dtype == torch.float64 and P.stride(1) == 1 and P.shape == (self.n_fn, self.n_fn)
        return kx_split_plan(self.ctx, P.data_ptr(), P.stride(0), kx_default_opts(**opts), budget)

    def worklist(self, a_filter=None) -> np.ndarray:
        return kx_get_worklist(self.ctx, a_filter)

    def order(self) -> np.ndarray:
        return kx_get_order(self.ctx, self.n_shell)

    def leaves(self):
        return kx_get_leaves(self.ctx)

    def profile(self) -> dict:
        return kx_get_profile(self.ctx)

    def norms(self, with_p: bool = True):
        return kx_get_norms(self.ctx, self.n_shell, with_p)

    def close(self):
        if getattr(self, "ctx", None):
            kx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchExchange:
    """A context for a batch of independent systems:
    ``BatchExchange(systems)(P) -> K`` with P and K packed (system y's
    n_y x n_y matrix at ``offsets[y]``, row-major) in 1-D float64 device
    tensors of ``size`` entries."""

    def __init__(self, systems, device: int = 0, leaf_max: int = 10, tau_ovlp: float = 0.0, stream=None):
        import torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.n_sys = len(systems)
        self.n_shell = [int(len(s.shell_l)) for s in systems]
        self.n_fn = [int(sum((l + 1) * (l + 2) // 2 for l in np.asarray(s.shell_l))) for s in systems]
        self.offsets = np.concatenate([[0], np.cumsum(np.asarray(self.n_fn, dtype=np.int64) ** 2)])
        self.shell_offsets = np.concatenate([[0], np.cumsum(self.n_shell)])
        self.ctx = kx_create_batch(systems, device, self.stream.cuda_stream)
        self.size = kx_packed_size(self.ctx)
        assert self.size == int(self.offsets[-1])
        kx_build_schwarz(self.ctx, tau_ovlp)
        kx_build_tree(self.ctx, leaf_max)

    def pack(self, mats):
        import torch
        return torch.cat([m.reshape(-1) for m in mats]).contiguous()

    def unpack(self, X):
        return [X[self.offsets[y]:self.offsets[y + 1]].view(self.n_fn[y], self.n_fn[y]) for y in range(self.n_sys)]

    def __call__(self, P, out=None, **opts):
        import torch
        assert P.is_cuda and P.dtype == torch.float64 and P.is_contiguous() and P.numel() == self.size
        K = out if out is not None else torch.empty_like(P)
        self.stats = kx_exchange_batch(self.ctx, P.data_ptr(), kx_default_opts(**opts), K.data_ptr())
        return K

    def host(self, P: np.ndarray, **opts) -> np.ndarray:
        K = np.zeros_like(P)
        self.stats = kx_exchange_batch_host(self.ctx, np.ascontiguousarray(P), kx_default_opts(**opts), K)
        return K

    def autotune(self, P, out=None, **opts):
        """One build that also tunes the class kernels' launch shapes."""
        import torch
        K = out if out is not None else torch.empty_like(P)
        self.stats, self.n_tuned = kx_autotune(self.ctx, P.data_ptr(), kx_default_opts(**opts), K.data_ptr())
        return K

    def plan(self, P, K, headroom: float = 0.25, **opts):
        """Captures a build reading P and writing K (static buffers) into a
        CUDA graph; ``replay()`` then rebuilds K from P's current contents."""
        self.stats = kx_graph_plan(self.ctx, P.data_ptr(), kx_default_opts(**opts), K.data_ptr(), headroom)
        self._graph_bufs = (P, K)
        return K

    def replay(self):
        self.stats = kx_graph_launch(self.ctx)
        return self._graph_bufs[1]

    def worklist(self) -> np.ndarray:
        return kx_get_worklist(self.ctx)

    def order(self) -> np.ndarray:
        return kx_get_order(self.ctx, int(self.shell_offsets[-1]))

    def leaves(self):
        return kx_get_leaves(self.ctx)

    def close(self) -> None:
        kx_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                kx_destroy(self.ctx)
        except Exception:
            pass
