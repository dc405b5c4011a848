#!/usr/bin/env python3
"""Benchmark of the screened exchange build on the (H2O)_64 workload.

One step = one complete exchange build K = sum (mu lam|nu sig) P_{lam sig}
(P norms and pyramid, pair tables, hextree traversal with the Eq. 8 metric
query, shell screen, ERI evaluation and contraction) of the seeded
(H2O)_64 cluster at 1 g/cm^3, medium basis (1984 functions, 1024 shells),
tau = 1e-10, leaves of at most 16 functions, replayed from one captured
CUDA graph (after an untimed split plan, autotuning build and capture).
The headline is the mixed-precision build: FP32 ERIs for the quartets with
beta <= split, double-word FP32 above it (FP64 for the classes without a
double-word kernel), the split chosen from an FP32 error budget.  Next to
it the line carries the plain FP64 build of the same system, the literal
split build (FP64 above the split) and the learned-culling build, each
with its max|dK| against the FP64 build.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
Under torchrun the ranks split one build by K row-block shards and sum K
with one all-reduce per step; ``--replicas`` gives every rank a whole
build instead.  ``--study`` runs the scaling sweep, the learned-culling
evaluation or the symmetry-case count instead of the benchmark.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "K-builds/s & ERI quartets/s vs plain FP64 GPU path at max|ΔK|≤1e-8"
UNIT = "K-builds/s"
WORKLOADS = ("water64", "water16", "batch256")
BATCH_TAU = 1e-8
TAU = 1e-10
SPLIT = 5e-4          # fixed split of the studies and the batch (measured max|dK| vs FP64: 3.0e-9 on (H2O)64)
SPLIT_BUDGET = 8e-9   # FP32 share of the 1e-8 bar: the benchmark build's split comes from kx_split_plan
BENCH_LEAF = 16       # leaf size of the benchmark builds (fastest of 10, 16, 20, 32 on (H2O)64)
L2_FLUSH_BYTES = 256 << 20
# headline precision: FP32 below the split, FP64 above ("mixed") or double-word FP32 above ("mixed_dw")
PRECISION = {"mixed": lambda kx: kx.KX_MIXED, "mixed_dw": lambda kx: kx.KX_MIXED_DW}
DTYPE = {"mixed": "f32+f64", "mixed_dw": "f32+dw32+f64"}

REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
           0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
           0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x100: "display_clocks_setting"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 3:
                continue
            try:
                s = float(parts[0])
                mx = float(parts[1])
                bits = int(parts[2], 16) if parts[2].startswith("0x") else int(parts[2])
            except ValueError:
                continue
            sm.append(s)
            for b, name in REASONS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_name(kx, ctx, s: int) -> str:
    """Name of the kernel that runs stream s (precision * 81 + class;
    precision 0 FP64, 1 FP32, 2 double-word FP32)."""
    cls = s % 81
    la, lb, lc, ld = cls // 27, (cls // 9) % 3, (cls // 3) % 3, cls % 3
    args = f"{la},{lb},{lc},{ld}"
    if s >= 162:
        return f"k_eri<{args},kx::dw>"
    if la + lb + lc + ld < 7:
        return f"k_eri<{args},{'double' if s < 81 else 'float'}>"
    variant = int(kx.kx_get_launch_shapes(ctx)[2][s])
    if s >= 81:
        return f"k_eri_bigp<{args}>" if variant == 1 else f"k_eri_big<{args}>"
    return {1: f"k_eri_big64<{args}>", 2: f"k_eri_big64p<{args}>"}.get(variant, f"k_eri_rolled<{args},double>")


def barrier(ws: int) -> None:
    """All ranks meet (no-op for one rank)."""
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest of every rank's x (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, ws: int, device) -> float:
    """The sum of every rank's x."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, seconds_max: float) -> float:
    """Whole-job throughput: the units of every rank over the slowest rank's time."""
    return ws * units_per_rank / seconds_max


PREC_NAME = ("fp64", "fp32", "dw")


def measured_alu_peaks(kx, device: int) -> dict:
    """TFLOP/s of the FP64 and FP32 FMA pipes and of double-word FP32
    multiply-adds, measured by the library's probes on this GPU."""
    return {"fp64": kx.kx_peak_probe(device, kx.KX_FP64) / 1e3, "fp32": kx.kx_peak_probe(device, kx.KX_MIXED) / 1e3,
            "dw": kx.kx_peak_probe(device, kx.KX_PROBE_DW) / 1e3}


def measured_peak(name: str):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f).get(name)
    except OSError:
        return None


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

ORACLE_ROW_SEED = 16   # the fixed seeded set of K-row shells the oracle samples


def oracle_row_set(sys_, n: int = 16, seed: int = ORACLE_ROW_SEED):
    """A fixed set of n K-row shells stratified by angular momentum: about
    n * (share of l among the shells) of each l, at least one of each l
    present, drawn with a fixed seed."""
    import numpy as np
    L = np.asarray(sys_.shell_l)
    rng = np.random.default_rng(seed)
    groups = []
    for l in sorted(set(L.tolist())):
        idx = np.nonzero(L == l)[0]
        k = max(1, int(round(n * len(idx) / len(L))))
        groups.append([int(x) for x in rng.choice(idx, size=min(k, len(idx)), replace=False)])
    # interleave the types (highest l first) so that any prefix mixes them
    rows = []
    for i in range(max(len(g) for g in groups)):
        rows += [g[i] for g in reversed(groups) if i < len(g)]
    return rows


def oracle_row_times(sys_, P, rows, leaf_max: int = 10, tau: float = None):
    """Seconds of the oracle's exact screened K rows of each shell in rows."""
    import oracle
    oracle.build()
    out = []
    for r in rows:
        t0 = time.perf_counter()
        oracle.exchange_screened(sys_, P, TAU if tau is None else tau, leaf_max=leaf_max, rows=[r])
        out.append((r, int(sys_.shell_l[r]), time.perf_counter() - t0))
    return out


def extrapolate_rows(sys_, times) -> float:
    """Seconds of a full build from row timings: for each angular momentum,
    its shell count times the mean time of its sampled rows (the mean of all
    sampled rows for a type that was not sampled)."""
    import numpy as np
    L = np.asarray(sys_.shell_l)
    allmean = float(np.mean([t for _, _, t in times]))
    total = 0.0
    for l in sorted(set(L.tolist())):
        ts = [t for _, ll, t in times if ll == l]
        total += int((L == l).sum()) * (float(np.mean(ts)) if ts else allmean)
    return total


def host_cpu() -> str:
    """CPU model and core count of this host (lscpu)."""
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        model = next((ln.split(":", 1)[1].strip() for ln in txt.splitlines() if ln.startswith("Model name")), "?")
        arch = next((ln.split(":", 1)[1].strip() for ln in txt.splitlines() if ln.startswith("Architecture")), "?")
    except (OSError, subprocess.SubprocessError):
        model, arch = "?", "?"
    return f"{os.cpu_count()} x {model} ({arch})"


def oracle_sample(sys_, P, n_rows: int, seed: int = 1, leaf_max: int = 10):
    """Exact screened K rows of the first n_rows shells of the fixed
    stratified row set, extrapolated per angular momentum to the full build;
    returns (seconds, K-builds/s, threads, description)."""
    import oracle
    rows = oracle_row_set(sys_)[:n_rows]
    times = oracle_row_times(sys_, P, rows, leaf_max)
    dt = sum(t for _, _, t in times)
    full = extrapolate_rows(sys_, times)
    desc = (f"oracle (FP64 C, OpenMP) screened exchange of {len(rows)} K-row shells (l = "
            f"{','.join(str(l) for _, l, _ in times)}) of {sys_.n_shell}, from a fixed seeded set stratified by "
            f"angular momentum ({dt:.1f} s), extrapolated per angular momentum to the full build; host "
            f"{host_cpu()}")
    return dt, 1.0 / full, oracle.num_threads(), desc


def oracle_batch_sample(systems, dens, n_sys: int, n_rows: int, seed: int = 1, leaf_max: int = 10):
    """Exact screened K rows of n_rows shells in each of n_sys sampled
    systems of a batch, extrapolated to every shell of every system."""
    import numpy as np

    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    picks = rng.choice(len(systems), size=n_sys, replace=False)
    t_all = 0.0
    est = 0.0
    for y in picks:
        s = systems[int(y)]
        rows = [int(x) for x in rng.choice(s.n_shell, size=n_rows, replace=False)]
        t0 = time.perf_counter()
        oracle.exchange_screened(s, dens[int(y)], BATCH_TAU, leaf_max=leaf_max, rows=rows)
        dt = time.perf_counter() - t0
        t_all += dt
        est += dt * s.n_shell / n_rows
    full = est * len(systems) / n_sys
    desc = (f"oracle (FP64 C, OpenMP) screened exchange of {n_rows} sampled K-row shells in each of {n_sys} "
            f"sampled clusters ({t_all:.1f} s), extrapolated to every shell of the {len(systems)} clusters")
    return t_all, len(systems) / full, oracle.num_threads(), desc


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import workloads as wl
    if args.workload == "batch256":
        systems, dens = wl.batch_workload()
        rates = []
        threads, desc = 1, ""
        for i in range(args.warmup + args.steps):
            dt, rate, threads, desc = oracle_batch_sample(systems, dens, 32, 4 * args.ref_rows, seed=100 + i,
                                                          leaf_max=args.leaf_max)
            if i >= args.warmup:
                rates.append(rate)
        v = statistics.mean(rates)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": batch_config(systems, "fp64", leaf_max=args.leaf_max),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    sys_, P = wl.workload(args.workload)
    # warm-up steps and timed steps, each a bounded sample of the workload:
    # step i times the next ref_rows shells of the fixed stratified row set
    import oracle
    rowset = oracle_row_set(sys_)
    timed = []
    for i in range(args.warmup + args.steps):
        rows = [rowset[(i * args.ref_rows + k) % len(rowset)] for k in range(args.ref_rows)]
        t = oracle_row_times(sys_, P, rows, args.leaf_max)
        if i >= args.warmup:
            timed += t
    v = 1.0 / extrapolate_rows(sys_, timed)
    threads = oracle.num_threads()
    desc = (f"oracle (FP64 C, OpenMP) screened exchange of K-row shells from a fixed set of {len(rowset)} "
            f"stratified by angular momentum, {args.ref_rows} per step ({len(timed)} timed rows, "
            f"{sum(t for _, _, t in timed):.1f} s), extrapolated per angular momentum to the full build; host "
            f"{host_cpu()}")
    single = single_thread_row(args.workload, min(timed, key=lambda x: x[2]), args.leaf_max)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(sys_, "fp64", args.workload, leaf_max=args.leaf_max),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
                             "single_thread": single},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def single_thread_row(workload: str, row, leaf_max: int, timeout_s: float = 120.0):
    """The cheapest timed K-row shell again, in a process whose OpenMP runs
    one thread: its time against the all-core time of the same row."""
    r, l, t_all = row
    code = ("import sys, time; sys.path.insert(0, %r); import oracle, workloads as wl; oracle.build(); "
            "s, P = wl.workload(%r); t0 = time.perf_counter(); "
            "oracle.exchange_screened(s, P, %r, leaf_max=%d, rows=[%d]); print(time.perf_counter() - t0)"
            % (ROOT, workload, TAU, leaf_max, r))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=timeout_s)
        t1 = float(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return {"row_shell": r, "l": l, "unavailable": f"single-thread run failed or exceeded {timeout_s:.0f} s"}
    return {"row_shell": r, "l": l, "seconds_1_thread": t1, "seconds_all_threads": t_all,
            "parallel_speedup": t1 / t_all}


def workload_config(sys_, precision, name, symmetric=True, leaf_max=10, split=SPLIT, parallelism="replicas"):
    nw = sys_.n_atom // 3
    return {"workload": f"(H2O){nw} water cluster at 1 g/cm^3, even-tempered medium basis "
                        f"({sys_.n_fn} functions, {sys_.n_shell} shells), tau=1e-10",
            "name": name,
            "n_fn": sys_.n_fn, "n_shell": sys_.n_shell, "tau": TAU, "leaf_max": leaf_max,
            "precision": precision, "split_threshold": split if precision.startswith("mixed") else None,
            "shell_screen": True, "symmetric": bool(symmetric),
            "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB buffer written)",
            "parallelism": parallelism}


def batch_config(systems, precision, symmetric=True, leaf_max=10):
    nw = [s.n_atom // 3 for s in systems]
    return {"workload": f"{len(systems)} independent water clusters of 4-48 molecules (drawn {min(nw)}-{max(nw)}), "
                        f"1 g/cm^3, small even-tempered basis (13 functions per water; "
                        f"{sum(s.n_fn for s in systems)} functions in all), each with its own density, "
                        f"tau={BATCH_TAU:g}",
            "name": "batch256", "systems": len(systems), "tau": BATCH_TAU, "leaf_max": leaf_max,
            "precision": precision, "split_threshold": SPLIT if precision.startswith("mixed") else None,
            "shell_screen": True, "symmetric": bool(symmetric),
            "launch": "one captured CUDA graph per batch build (autotuned class-kernel shapes)",
            "l2": "inputs larger than L2 (packed P and K 297 MB each), and a 256 MB buffer written between steps",
            "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_batch(args):
    """The batched workload: 256 clusters per step, replayed from one CUDA graph."""
    import numpy as np
    import torch

    import paper_1401_6961_gb300 as kx
    import workloads as wl

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kx.load()
    systems, dens = wl.batch_workload()
    stream = torch.cuda.current_stream(dev)
    bx = kx.BatchExchange(systems, device=local, stream=stream, leaf_max=args.leaf_max)
    Pd = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).to(dev)
    Kd = torch.empty_like(Pd)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    sym = 0 if args.no_symmetric else 1
    mixed = dict(tau=BATCH_TAU, precision=PRECISION[args.precision](kx), split_threshold=SPLIT, symmetric=sym)


    # set-up (untimed): launch-shape autotuning, then the captured plan
    bx.autotune(Pd, out=Kd, **mixed)
    n_tuned = bx.n_tuned
    bx.plan(Pd, Kd, headroom=0.25, **mixed)
    for _ in range(args.warmup):
        bx.replay()
    torch.cuda.synchronize(dev)
    barrier(ws)
    torch.cuda.synchronize(dev)
    evs = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bx.replay()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
    barrier(ws)
    st = bx.stats
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws, dev)
    ms_step = ms / args.steps
    nsys = len(systems)
    value = job_rate(nsys, ws, ms_step * 1e-3)
    Kmix = Kd.clone()

    # per-class profile of an eager mixed build with the same launch shapes
    bx(Pd, out=Kd, profile=1, **mixed)
    prof = kx.kx_get_profile(bx.ctx)
    ste = bx.stats
    s_dom = int(np.argmax(prof["ms"]))
    prec_dom = PREC_NAME[s_dom // 81]
    cls = s_dom % 81
    la, lb, lc, ld = cls // 27, (cls // 9) % 3, (cls // 3) % 3, cls % 3
    peaks = measured_alu_peaks(kx, local)
    peak = peaks[prec_dom]
    achieved = prof["flops"][s_dom] / (prof["ms"][s_dom] * 1e-3) / 1e12

    fp64 = None
    diff = None
    if args.fp64_steps > 0:
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            bx(Pd, out=Kd, tau=BATCH_TAU, precision=kx.KX_FP64, symmetric=sym)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = max_over_ranks(e0.elapsed_time(e1), ws, dev) / args.fp64_steps
        diff = float((Kmix - Kd).abs().max().item())
        fp64 = {"value": ws * nsys * 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
                "warmup": 0, "launch": "eager", "quartets_per_s": ws * bx.stats.n_shell_quartets / (ms64 * 1e-3)}

    e2e = None
    if args.e2e_steps > 0:
        Ph = torch.from_numpy(np.concatenate([d.ravel() for d in dens])).pin_memory().numpy()
        Kh = torch.empty(Ph.shape[0], dtype=torch.float64).pin_memory().numpy()
        o = kx.kx_default_opts(**mixed)
        kx.kx_exchange_batch_host(bx.ctx, Ph, o, Kh)
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            kx.kx_exchange_batch_host(bx.ctx, Ph, o, Kh)
        dt = max_over_ranks(time.perf_counter() - t0, ws, dev)
        e2e = {"value": ws * nsys * args.e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * Ph.shape[0],
               "d2h_bytes_per_step": 8 * Ph.shape[0], "launch": "eager (kx_exchange_batch_host)"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        dt, rate, thr, desc = oracle_batch_sample(systems, dens, 32, 4 * args.ref_rows, leaf_max=args.leaf_max)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": batch_config(systems, args.precision, sym, args.leaf_max),
            "quartets_per_s": ws * st.n_shell_quartets / (ms_step * 1e-3),
            "shell_quartets": st.n_shell_quartets, "leaf_quartets": st.n_leaf_quartets,
            "shell_quartets_fp64": st.n_shell_quartets_fp64, "shell_quartets_dw": st.n_shell_quartets_dw,
            "stages_ms_eager": {"norms": ste.ms_norms, "traverse": ste.ms_traverse, "expand": ste.ms_expand,
                                "eri": ste.ms_eri, "total": ste.ms_total},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": kernel_name(kx, bx.ctx, s_dom),
                         "measured": "CUDA events around each launch of that kernel in an eager profiled build "
                                     "of the same batch (a graph replay cannot be split by events)",
                         "peak_source": f"measured probe ({prec_dom}), kx_peak_probe"},
            "fp64_plain": fp64,
            "speedup_vs_fp64_plain": (value / fp64["value"]) if fp64 else None,
            "max_abs_dK_vs_fp64": diff,
            "streams_tuned": n_tuned,
            "e2e": e2e,
            "gpu_launches": int(st.n_launches) * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    bx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def learned_leg(kx, ex, Pd, K64, stream, opts, leaf_max, ws):
    """The learned-culling build of the benchmark system next to the plain
    mixed build: training traces of medium-basis (H2O)4 and (H2O)8, margin
    from a held-out (H2O)12 (99.9 % quantile of the residual), then one
    warm-up and one timed culled build."""
    import torch

    import workloads as wl
    from paper_1401_6961_gb300 import learned

    tau = opts["tau"]
    t0 = time.perf_counter()

    def tr_of(n_w, seed, samples):
        s = wl.water_cluster(n_w, seed, "medium")
        e = kx.Exchange(s, device=ex.device, stream=stream, leaf_max=leaf_max)
        t = learned.traces(e, torch.from_numpy(wl.density(s, 1000 + seed)).to(Pd.device), tau,
                           max_samples=samples, seed=1)
        e.close()
        return t
    tr = tr_of(4, 104, 20000) + tr_of(8, 108, 20000)
    model = learned.train(tr, epochs=200, lr=3e-3, batch=4096)
    model = learned.calibrate(model, tr_of(12, 112, 20000), q=0.999)
    set_up_s = time.perf_counter() - t0
    K = torch.empty_like(Pd)
    learned.learned_exchange(ex, Pd, model, tau, K=K, **{k: v for k, v in opts.items() if k != "tau"})
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, info = learned.learned_exchange(ex, Pd, model, tau, K=K, **{k: v for k, v in opts.items() if k != "tau"})
    e1.record(stream)
    torch.cuda.synchronize(Pd.device)
    ms = e0.elapsed_time(e1)
    return {"value": ws * 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "steps": 1,
            "launch": "eager (traversal, features, BF16 inference, cull, ERI stage)",
            "leaf_quartets": info["leaf_quartets"], "leaf_quartets_kept": info["leaf_quartets_kept"],
            "leaf_quartets_cullable": info["cullable"], "shell_quartets": info["shell_quartets"],
            "max_abs_dK_vs_fp64": float((K - K64).abs().max().item()),
            "training": {"traces": int(len(tr.targets)), "loss_first": model.losses[0],
                         "loss_last": model.losses[-1], "margin_decades": model.margin,
                         "set_up_s": set_up_s}}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1401_6961_gb300 as kx
    import workloads as wl

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kx.load()
    sys_, P = wl.workload(args.workload)
    stream = torch.cuda.current_stream(dev)
    ex = kx.Exchange(sys_, device=local, stream=stream, leaf_max=args.leaf_max)
    n = sys_.n_fn
    Pd = torch.from_numpy(P).to(dev)
    Kd = torch.empty((n, n), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    sym = 0 if args.no_symmetric else 1
    prec = PRECISION[args.precision](kx)
    # the split: from the FP32 error budget (kx_split_plan, untimed set-up), or fixed
    if args.split_budget > 0:
        sp = ex.split_plan(Pd, args.split_budget, tau=TAU, symmetric=sym)
        split = sp.split_used
        split_info = {"budget": args.split_budget, "split": split, "fp32_err_estimate_5sigma": sp.fp32_err_estimate,
                      "fp32_err_bound": sp.fp32_err_bound, "how": "kx_split_plan: per-class FP32 error constants, "
                      "sampled K shell blocks, largest tau*2^k whose 5-sigma estimate fits the budget"}
    else:
        split = SPLIT
        split_info = {"split": split, "how": "fixed"}
    mixed = dict(tau=TAU, precision=prec, split_threshold=split, profile=1, symmetric=sym)
    plain = dict(tau=TAU, precision=kx.KX_FP64, profile=1, symmetric=sym)
    # several ranks: each builds the K rows of its balanced row-block shard
    # (kx_row_work / kx_shard_bounds; every rank computes the same plan) and
    # one sum over the ranks assembles K inside the timed step
    sharded = ws > 1 and not args.replicas
    if sharded:
        from paper_1401_6961_gb300 import shard
        bounds = shard.plan(ex, Pd, ws, tau=TAU, precision=prec, split_threshold=split, symmetric=sym)
        rows = dict(row_leaf_lo=int(bounds[rank]), row_leaf_hi=int(bounds[rank + 1]))
        mixed.update(rows)
        plain.update(rows)

    def assemble(K):
        if sharded:
            shard.assemble(K)


    def timed_steps(opts, steps):
        evs = []
        launches = 0
        prof = None
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ex(Pd, out=Kd, **opts)
            e1.record(stream)
            evs.append((e0, e1))
            launches += ex.stats.n_launches
            p = ex.profile()
            if prof is None:
                prof = {k: v.astype(float).copy() for k, v in p.items()}
            else:
                for k in prof:
                    prof[k] += p[k]
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, launches, prof

    # set-up (untimed): launch-shape autotuning of the class kernels, then the
    # captured build (one CUDA graph per exchange build)
    nomix = {k: v for k, v in mixed.items() if k != "profile"}
    ex.autotune(Pd, out=Kd, **nomix)
    n_tuned = ex.n_tuned
    ex.plan(Pd, Kd, headroom=0.25, **nomix)
    for _ in range(args.warmup):
        ex.replay()
    torch.cuda.synchronize(dev)
    barrier(ws)
    torch.cuda.synchronize(dev)
    evs = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ex.replay()
            assemble(Kd)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
    barrier(ws)
    st = ex.stats
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws, dev)
    ms_step = ms / args.steps
    # replicas: every rank built a whole K; shards: the ranks built one K together
    value = job_rate(1, 1 if sharded else ws, ms_step * 1e-3)
    quartets = st.n_shell_quartets
    # every rank's quartets: a shard's own, a replica's whole build
    quartets_all = sum_over_ranks(float(quartets), ws, dev)
    launches = int(st.n_launches) * args.steps
    Kmix = Kd.clone()

    # the same build run eagerly with every class launch timed by CUDA events
    # (per-kernel times cannot be taken inside a graph replay): stage times
    # and the roofline of the dominant class kernel
    torch.cuda.synchronize(dev)
    ms_e, _, prof = timed_steps(mixed, max(1, args.eager_steps))
    ms_e = max_over_ranks(ms_e, ws, dev) / max(1, args.eager_steps)
    ste = ex.stats

    # roofline of the dominant ERI class kernel over the timed steps
    s_dom = int(np.argmax(prof["ms"]))
    prec_dom = PREC_NAME[s_dom // 81]
    cls = s_dom % 81
    la, lb, lc, ld = cls // 27, (cls // 9) % 3, (cls // 3) % 3, cls % 3
    dom_ms = prof["ms"][s_dom]
    dom_launch = max(prof["launches"][s_dom], 1)
    achieved = prof["flops"][s_dom] / (dom_ms * 1e-3) / 1e12
    peaks = measured_alu_peaks(kx, local)
    peak64, peak32, peakdw = peaks["fp64"], peaks["fp32"], peaks["dw"]
    peak = peaks[prec_dom]
    eri_ms = float(prof["ms"].sum())
    # every class stream of the eager builds, on stderr
    streams = []
    for s_ in range(kx.NSTREAM):
        if prof["ms"][s_] > 0:
            c_ = s_ % 81
            streams.append({"stream": s_, "class": "({}{}|{}{})".format(*("spd"[x] for x in (
                c_ // 27, (c_ // 9) % 3, (c_ // 3) % 3, c_ % 3))), "precision": PREC_NAME[s_ // 81],
                "kernel": kernel_name(kx, ex.ctx, s_), "ms": float(prof["ms"][s_]), "quartets": int(prof["n"][s_]),
                "tflops": float(prof["flops"][s_] / (prof["ms"][s_] * 1e-3) / 1e12)})
    print(json.dumps({"eri_streams": streams}), file=sys.stderr, flush=True)
    # the ten costliest class streams of the eager builds
    top = []
    for s_ in np.argsort(-prof["ms"])[:10]:
        s_ = int(s_)
        if prof["ms"][s_] <= 0:
            break
        c_ = s_ % 81
        top.append({"class": "({}{}|{}{})".format(*("spd"[x] for x in (c_ // 27, (c_ // 9) % 3, (c_ // 3) % 3,
                                                                       c_ % 3))),
                    "precision": PREC_NAME[s_ // 81], "kernel": kernel_name(kx, ex.ctx, s_),
                    "ms": float(prof["ms"][s_]) / max(1, args.eager_steps),
                    "quartets": int(prof["n"][s_]) // max(1, args.eager_steps),
                    "tflops": float(prof["flops"][s_] / (prof["ms"][s_] * 1e-3) / 1e12)})
    eri_flops64 = float(prof["flops"][:81].sum())
    eri_flops32 = float(prof["flops"][81:162].sum())
    eri_flopsdw = float(prof["flops"][162:].sum())
    # step-level ALU fraction: the time the step's algorithmic FLOPs need at
    # the measured peak of the pipe each runs on, over the measured step
    steps_e = max(1, args.eager_steps)
    floor_ms = 1e3 * (eri_flops64 / (peak64 * 1e12) + eri_flops32 / (peak32 * 1e12)
                      + eri_flopsdw / (peakdw * 1e12)) / steps_e

    # plain FP64 build of the same system (the speed-up denominator)
    # plain FP64 build of the same system, captured and replayed the same way
    fp64 = None
    if args.fp64_steps > 0:
        ex.plan(Pd, Kd, headroom=0.25, **{k: v for k, v in plain.items() if k != "profile"})
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            ex.replay()
            assemble(Kd)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = max_over_ranks(e0.elapsed_time(e1), ws, dev) / args.fp64_steps
        s64 = ex.stats
        diff = float((Kmix - Kd).abs().max().item())
        K64 = Kd.clone()
        fp64 = {"value": (1 if sharded else ws) * 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64,
                "steps": args.fp64_steps, "warmup": 0, "launch": "captured graph, replayed",
                "quartets_per_s": ws * s64.n_shell_quartets / (ms64 * 1e-3),
                "build_tflops_fp64": s64.flops_fp64 / (ms64 * 1e-3) / 1e12,
                "build_frac_of_fp64_peak": s64.flops_fp64 / (ms64 * 1e-3) / 1e12 / peak64}
    else:
        diff = None

    # the contract's literal split precision (FP64 above the split), captured
    # and replayed the same way, when the headline uses double words there
    lit = None
    if args.precision != "mixed" and args.fp64_steps > 0:
        ex.plan(Pd, Kd, headroom=0.25, **dict(nomix, precision=kx.KX_MIXED))
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            ex.replay()
            assemble(Kd)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        msl = max_over_ranks(e0.elapsed_time(e1), ws, dev) / args.fp64_steps
        lit = {"value": (1 if sharded else ws) * 1e3 / msl, "unit": UNIT, "ms_per_step": msl, "steps": args.fp64_steps,
               "precision": "fp32 below the split, fp64 above", "shell_quartets_fp64": ex.stats.n_shell_quartets_fp64,
               "launch": "captured graph, replayed",
               "max_abs_dK_vs_fp64": float((Kd - K64).abs().max().item()) if fp64 else None}

    # mixed precision + learned culling (the target build of the learned
    # direction): the network is trained and its margin calibrated on small
    # clusters of the same basis at the same tau and leaf size (untimed),
    # then the culled build -- traversal, features, BF16 inference, cull and
    # the ERI stage -- runs eagerly
    lrn = None
    if args.learned and not sharded and args.fp64_steps > 0:
        lrn = learned_leg(kx, ex, Pd, K64, stream, nomix, args.leaf_max, ws)
        lrn["speedup_vs_fp64_plain"] = lrn["value"] / fp64["value"]
        lrn["shell_quartets_plain_mixed"] = int(quartets)

    # end to end through the host-buffer entry point (pinned host P and K)
    e2e = None
    if args.e2e_steps > 0:
        Ph = torch.from_numpy(P).pin_memory().numpy()
        Kh = torch.empty((n, n), dtype=torch.float64).pin_memory().numpy()
        ex.host(Ph, tau=TAU, precision=prec, split_threshold=split, symmetric=sym)
        barrier(ws)
        t0 = time.perf_counter()
        ho = {k: v for k, v in nomix.items()}
        for _ in range(args.e2e_steps):
            kx.kx_exchange_host(ex.ctx, Ph, kx.kx_default_opts(**ho), Kh)
        dt = max_over_ranks(time.perf_counter() - t0, ws, dev)
        e2e = {"value": (1 if sharded else ws) * args.e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * n * n,
               "d2h_bytes_per_step": 8 * n * n}
        if sharded:
            e2e["note"] = "each rank copies P in and its shard's K out; the sum over ranks is not in this figure"

    cpu = None
    if rank == 0 and not args.no_cpu:
        # the first three shells of the fixed row set: one of each angular momentum
        dt, rate, thr, desc = oracle_sample(sys_, P, 3, leaf_max=args.leaf_max)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": workload_config(sys_, args.precision, args.workload, sym, args.leaf_max, split,
                                      "row-block shards, one all-reduce of K per step" if sharded else "replicas"),
            "split": split_info,
            "quartets_per_s": quartets_all / (ms_step * 1e-3),
            "shell_quartets": quartets, "leaf_quartets": st.n_leaf_quartets,
            "shell_quartets_fp64": st.n_shell_quartets_fp64, "shell_quartets_dw": st.n_shell_quartets_dw,
            "launch": "one captured CUDA graph per build (kx_graph_plan / kx_graph_launch), autotuned "
                      f"class-kernel shapes ({n_tuned} streams tuned)",
            "eager": {"value": ws * 1e3 / ms_e, "unit": UNIT, "ms_per_step": ms_e,
                      "steps": max(1, args.eager_steps), "launches_per_step": int(ste.n_launches),
                      "profile": "CUDA events around every class launch"},
            "stages_ms_eager": {"norms": ste.ms_norms, "traverse": ste.ms_traverse, "expand": ste.ms_expand,
                                "eri": ste.ms_eri},
            "shell_screen": {"candidates": int(ste.n_candidates), "ms_eager": ste.ms_expand,
                             "candidates_per_s": ste.n_candidates / max(ste.ms_expand * 1e-3, 1e-12),
                             "kept": int(ste.n_shell_quartets),
                             "unit": "shell quartets of the kept leaf quartets, each tested against Eq. 8 "
                                     "(count and write passes)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": kernel_name(kx, ex.ctx, s_dom),
                         "launches": int(prof["launches"][s_dom]),
                         "ms_per_launch": dom_ms / dom_launch,
                         "measured": "CUDA events on the launching stream around each launch of that kernel, "
                                     "in the eager builds of the same system that follow the timed replays",
                         "peak_source": f"measured probe ({prec_dom}), kx_peak_probe"},
            "eri_classes_top": top,
            "eri_stage": {"ms_per_step": eri_ms / max(1, args.eager_steps),
                          "tflops": (eri_flops64 + eri_flops32 + eri_flopsdw) / (eri_ms * 1e-3) / 1e12,
                          "flops_fp64_per_step": eri_flops64 / steps_e,
                          "flops_fp32_per_step": eri_flops32 / steps_e,
                          "flops_dw_per_step": eri_flopsdw / steps_e,
                          "peak_fp64_tflops": peak64, "peak_fp32_tflops": peak32, "peak_dw_tflops": peakdw},
            "step_roofline": {"bound": "alu", "floor_ms": floor_ms, "ms_per_step": ms_step,
                              "frac": floor_ms / ms_step, "eri_frac": floor_ms / (eri_ms / steps_e),
                              "how": "algorithmic FLOPs of each precision at its measured peak (kx_peak_probe: "
                                     "FP64 and FP32 FMA pipes, double-word FMA chains), summed, over the "
                                     "replayed step and over the ERI stage of the eager step"},
            "fp64_plain": fp64,
            "speedup_vs_fp64_plain": (value / fp64["value"]) if fp64 else None,
            "max_abs_dK_vs_fp64": diff,
            "mixed_fp64_above_split": lit,
            "mixed_learned": lrn,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ex.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()



# ---------------------------------------------------------------------------
# studies (not the benchmark line): the scaling sweep and the learned culling
# ---------------------------------------------------------------------------

SWEEP_N = (64, 128, 256, 512)
SWEEP_TAU = (1e-10, 1e-8, 1e-6)
SWEEP_BUILD_S = 200.0     # time a mixed build only when the count predicts at most this many seconds
SWEEP_FP64_S = 60.0       # and the FP64 build of the same point at most this many
SWEEP_MAX_SHELL_Q = 4e12  # counts (traversal + count pass of the screen) stay within about a minute
SWEEP_MAX_LEAF_Q = 1.5e10  # and the frontier before the last level within a few tens of GB
SWEEP_GROWTH = 2.5        # predicted survivors grow as n_fn^2.5 (measured: 1.7-2.6)
RATE_MIXED, RATE_FP64 = 8e9, 1e9   # shell quartets/s of the (H2O)64 builds, for that prediction


def _event_ms(stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def run_sweep(args):
    """Scaling sweep (H2O)_n, n = 64..512 at 1 g/cm^3, tau in {1e-10, 1e-8,
    1e-6}: survivors of the plain method (every K block) against n, their
    growth exponent next to the N lg N trend, and timed mixed / FP64 builds
    (symmetric) where they fit the time cap."""
    import numpy as np
    import torch

    import paper_1401_6961_gb300 as kx
    import workloads as wl

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    kx.load()
    stream = torch.cuda.current_stream(dev)
    bases = [b.strip() for b in args.sweep_bases.split(",") if b.strip()]
    ns = [int(x) for x in args.sweep_n.split(",")]
    taus_all = [float(x) for x in args.sweep_taus.split(",")]
    rows = []
    last = {}
    for basis in bases:
        for nw in ns:
            sys_ = wl.water_sweep(nw, basis)
            taus = []
            for tau in taus_all:
                prev = last.get((basis, tau))
                if prev is not None:
                    # growth from the previous size, above the measured exponents
                    g = (sys_.n_fn / prev[0]) ** SWEEP_GROWTH
                    if prev[1] * g > SWEEP_MAX_SHELL_Q or prev[2] * g > SWEEP_MAX_LEAF_Q:
                        rows.append({"basis": basis, "n_water": nw, "n_fn": sys_.n_fn, "tau": tau,
                                     "skipped": f"predicted more than {SWEEP_MAX_SHELL_Q:.0e} shell quartets or "
                                                f"{SWEEP_MAX_LEAF_Q:.0e} leaf quartets"})
                        continue
                taus.append(tau)
            if not taus:
                continue
            P = wl.density(sys_, 5000 + nw)
            t0 = time.perf_counter()
            ex = kx.Exchange(sys_, device=0, stream=stream, leaf_max=args.leaf_max)
            setup_s = time.perf_counter() - t0
            Pd = torch.from_numpy(P).to(dev)
            del P
            K = torch.empty_like(Pd)
            for tau in taus:
                mixed = dict(tau=tau, precision=PRECISION[args.precision](kx), split_threshold=SPLIT)
                ms_c, full = _event_ms(stream, lambda: ex.count(Pd, symmetric=0, **mixed))
                last[(basis, tau)] = (sys_.n_fn, full.n_shell_quartets, full.n_leaf_quartets)
                half = ex.count(Pd, symmetric=1, **mixed)
                row = {"basis": basis, "n_water": nw, "n_fn": sys_.n_fn, "n_shell": sys_.n_shell, "tau": tau,
                       "leaf_quartets": full.n_leaf_quartets, "shell_quartets": full.n_shell_quartets,
                       "candidates": full.n_candidates, "shell_quartets_symmetric": half.n_shell_quartets,
                       "shell_quartets_fp64_symmetric": half.n_shell_quartets_fp64,
                       "count_ms": ms_c, "setup_s": setup_s}
                q = half.n_shell_quartets
                if q / RATE_MIXED <= SWEEP_BUILD_S:
                    ex(Pd, out=K, symmetric=1, **mixed)            # warm-up
                    ms, _ = _event_ms(stream, lambda: ex(Pd, out=K, symmetric=1, **mixed))
                    row["mixed_ms"] = ms
                    row["mixed_quartets_per_s"] = q / (ms * 1e-3)
                    if q / RATE_FP64 <= SWEEP_FP64_S:
                        Km = K.clone()
                        ms64, _ = _event_ms(stream, lambda: ex(Pd, out=K, symmetric=1, tau=tau,
                                                               precision=kx.KX_FP64))
                        row["fp64_ms"] = ms64
                        row["speedup_mixed_vs_fp64"] = ms64 / ms
                        row["max_abs_dK_mixed_vs_fp64"] = float((Km - K).abs().max().item())
                        del Km
                rows.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
            ex.close()
            del Pd, K
            torch.cuda.empty_cache()
    # growth exponents: least squares of log(survivors) against log(n_fn)
    fits = []
    for basis in bases:
        for tau in taus_all:
            pts = [(r["n_fn"], r["shell_quartets"], r["leaf_quartets"]) for r in rows
                   if r["basis"] == basis and r["tau"] == tau and r.get("shell_quartets", 0) > 0]
            if len(pts) < 2:
                continue
            x = np.log([p[0] for p in pts])
            fits.append({"basis": basis, "tau": tau,
                         "exponent_shell_quartets": float(np.polyfit(x, np.log([p[1] for p in pts]), 1)[0]),
                         "exponent_leaf_quartets": float(np.polyfit(x, np.log([p[2] for p in pts]), 1)[0]),
                         "exponent_n_lg_n": float(np.polyfit(x, np.log([p[0] * math.log2(p[0]) for p in pts]),
                                                             1)[0])})
    print(json.dumps({"study": "sweep", "workload": "(H2O)_n at 1 g/cm^3, n = " + ",".join(map(str, ns)),
                      "precision": args.precision, "split_threshold": SPLIT, "leaf_max": args.leaf_max,
                      "points": rows, "fits": fits}),
          flush=True)


def run_learned(args):
    """Learned culling: train the network on traces of small water clusters,
    two clusters of the batched workload and a short alkane, then compare on
    alkanes C_nH_2n+2 and (H2O)_256 (small basis, tau = 1e-8) the plain FP64
    build, the plain mixed build and the mixed build with learned culling."""
    import torch

    import paper_1401_6961_gb300 as kx
    import workloads as wl
    from paper_1401_6961_gb300 import learned

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    kx.load()
    stream = torch.cuda.current_stream(dev)
    tau = 1e-8
    w8, c6 = wl.water_cluster(8, 8, "small"), wl.alkane(6, 66, "small")
    train_sets = [("water4", *wl.workload("water4")), ("(H2O)8", w8, wl.density(w8, 808)),
                  ("C6H14", c6, wl.density(c6, 812))]
    batch_sys, batch_dens = wl.batch_workload()
    for i in (0, 1):
        train_sets.append((f"batch cluster {i} ({batch_sys[i].n_atom // 3} waters)", batch_sys[i], batch_dens[i]))
    tr = None
    t0 = time.perf_counter()
    for name, s, P in train_sets:
        ex = kx.Exchange(s, device=0, stream=stream)
        t = learned.traces(ex, torch.from_numpy(P).to(dev), tau, max_samples=20000, seed=1)
        tr = t if tr is None else tr + t
        ex.close()
    t_tr = time.perf_counter() - t0
    t0 = time.perf_counter()
    model = learned.train(tr, epochs=args.epochs, lr=3e-3, batch=4096)
    t_train = time.perf_counter() - t0
    evals = []
    targets = [(f"C{n}H{2 * n + 2}", wl.alkane(n, 6000 + n), 7000 + n) for n in (10, 20, 40, 80)]
    s256 = wl.water_sweep(256, "small")
    targets.append(("(H2O)256", s256, 5256))
    for name, s, pseed in targets:
        Pd = torch.from_numpy(wl.density(s, pseed)).to(dev)
        ex = kx.Exchange(s, device=0, stream=stream)
        K64 = torch.empty_like(Pd)
        ex(Pd, out=K64, tau=tau)                                            # warm-up
        ms64, _ = _event_ms(stream, lambda: ex(Pd, out=K64, tau=tau))
        st64 = ex.stats
        Km = torch.empty_like(Pd)
        msm, _ = _event_ms(stream, lambda: ex(Pd, out=Km, tau=tau, precision=kx.KX_MIXED, split_threshold=SPLIT))
        stm = ex.stats
        Kl = torch.empty_like(Pd)
        learned.learned_exchange(ex, Pd, model, tau, K=Kl, precision=kx.KX_MIXED, split_threshold=SPLIT)
        msl, (_, info) = _event_ms(stream, lambda: learned.learned_exchange(
            ex, Pd, model, tau, K=Kl, precision=kx.KX_MIXED, split_threshold=SPLIT))
        row = {"system": name, "n_fn": s.n_fn, "tau": tau,
               "leaf_quartets": st64.n_leaf_quartets, "leaf_quartets_learned": info["leaf_quartets_kept"],
               "leaf_quartets_cullable": info["cullable"],
               "shell_quartets": stm.n_shell_quartets, "shell_quartets_learned": info["shell_quartets"],
               "fp64_ms": ms64, "mixed_ms": msm, "learned_mixed_ms": msl,
               "speedup_mixed": ms64 / msm, "speedup_learned_mixed": ms64 / msl,
               "max_abs_dK_mixed_vs_fp64": float((Km - K64).abs().max().item()),
               "max_abs_dK_learned_vs_fp64": float((Kl - K64).abs().max().item())}
        evals.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
        ex.close()
    print(json.dumps({"study": "learned", "tau": tau, "split_threshold": SPLIT,
                      "training": {"systems": [t[0] for t in train_sets], "traces": int(len(tr.targets)),
                                   "epochs": args.epochs, "loss_first": model.losses[0],
                                   "loss_last": model.losses[-1], "residual_std_decades": model.residual_std,
                                   "trace_s": t_tr, "train_s": t_train},
                      "evaluation": evals}), flush=True)


def run_symmetry(args):
    """The symmetry cases of Eqs. 9-10 among the kept leaf quartets of
    (H2O)_n builds (medium basis, tau = 1e-10, every K block): the shares of
    full 4-fold blocks, blocks with coinciding index blocks and sparse
    blocks, the kept quartets per canonical integral block, the share of
    the ERI FLOPs that does not involve P, and the bound that gives on what
    the further index swaps could save over the K-transpose half."""
    import numpy as np
    import torch

    import paper_1401_6961_gb300 as kx
    import workloads as wl
    from paper_1401_6961_gb300 import symmetry

    torch.cuda.set_device(0)
    kx.load()
    rows = []
    for nw in [int(x) for x in args.sym_n.split(",")]:
        sys_ = wl.water_sweep(nw, "medium") if nw != 64 else wl.water64(2)
        P = wl.density(sys_, 5000 + nw) if nw != 64 else wl.workload("water64")[1]
        ex = kx.Exchange(sys_, device=0, leaf_max=args.leaf_max)
        Pd = torch.from_numpy(P).cuda()
        ex(Pd, tau=TAU, symmetric=0, keep_worklist=1)
        work = ex.worklist()
        occ = symmetry.occurrence_counts(work)
        # ERI FLOPs of the symmetric build by class, and their integral part
        ex(Pd, tau=TAU, symmetric=1, profile=1)
        prof = ex.profile()
        n_cls = prof["n"][:81] + prof["n"][81:162] + prof["n"][162:]
        f_int = symmetry.integral_share(n_cls)
        tasks_sym = int((work[:, 0] <= work[:, 2]).sum())
        reuse = occ["blocks"] / tasks_sym
        row = {"n_water": nw, "n_fn": sys_.n_fn, "leaf_max": args.leaf_max, "tau": TAU, **occ,
               "share_full": occ["full"] / occ["blocks"], "share_coincident": occ["coincident"] / occ["blocks"],
               "share_sparse": occ["sparse"] / occ["blocks"], "tasks_symmetric": tasks_sym,
               "canonical_blocks_per_symmetric_task": reuse, "eri_integral_flop_share": f_int,
               "bound_eri_flops_saved": f_int * (1.0 - reuse)}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
        ex.close()
    print(json.dumps({"study": "symmetry", "points": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="water64",
                    help="water64 is the benchmark; water16 is a small case for profiling; batch256 is the "
                         "batched workload (256 clusters per step, captured graph)")
    ap.add_argument("--precision", choices=sorted(PRECISION), default="mixed_dw",
                    help="headline build: FP32 below the split and FP64 (mixed) or double-word FP32 (mixed_dw) above")
    ap.add_argument("--split-budget", type=float, default=SPLIT_BUDGET,
                    help="FP32 error budget of the split planner; 0 = the fixed split")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--eager-steps", type=int, default=1, help="profiled eager builds after the timed replays")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-rows", type=int, default=2, help="K-row shells per oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned-culling build of the benchmark system")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun, every rank builds the whole K instead of its row-block shard")
    ap.add_argument("--no-symmetric", action="store_true",
                    help="build every K block instead of the A <= C half and its mirror")
    ap.add_argument("--leaf-max", type=int, default=BENCH_LEAF,
                    help="bisection leaf size in functions (Eq. 1); the paper's CPU code used 10")
    ap.add_argument("--sym-n", default="16,32,64", help="water cluster sizes of the symmetry study")
    ap.add_argument("--study", choices=["sweep", "learned", "symmetry"], default=None,
                    help="instead of the benchmark line: the (H2O)_n scaling sweep, or the learned-culling "
                         "evaluation (one JSON line each, per-point lines on stderr)")
    ap.add_argument("--sweep-n", default=",".join(map(str, SWEEP_N)))
    ap.add_argument("--sweep-bases", default="medium,small")
    ap.add_argument("--sweep-taus", default=",".join(map(str, SWEEP_TAU)))
    ap.add_argument("--epochs", type=int, default=300)
    args = ap.parse_args()
    if args.study == "sweep":
        run_sweep(args)
    elif args.study == "symmetry":
        run_symmetry(args)
    elif args.study == "learned":
        run_learned(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
