"""Benchmark: preconditioned FGMRES solves/s on the 512x512 inviscid-like grid.

One step = one full solve through the C ABI: block ILU(0) built from A by 6
sweeps (FP32 factors, refined FP32 inversion), FGMRES(30) to a relative residual of
1e-6 with 4+4 triangular sweeps per preconditioner application, FP64 SpMV,
Arnoldi and Givens.  The pattern is analysed once (values change per
pseudo-time step, the pattern does not); A and b are resident in HBM when the
timed region starts.  A (268 MB) is larger than L2, so no L2 flush is needed.

Also reported: the same solve end to end with A and b copied from pinned host
memory and x copied back every step ("e2e"; double-buffered, the next step's
inputs stream in on a copy stream while the current step solves); per-kernel
achieved bandwidth
against the measured HBM copy peak ("roofline", "kernels"); the CPU oracle's
solve rate on the host ("cpu_baseline"); p50/p99 solve latency; other
precision/mode variants.  ``--impl reference`` times the CPU oracle instead.
Under torchrun every rank solves its own replica (the systems are independent),
value = solves of all ranks / max wall time over ranks.  Other workloads:
--batched, --serving, --viscous, --continuation, --scalar, --kernels-only.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "inviscid_512x512"
BUILD_SWEEPS, APPLY_SWEEPS, RESTART, RTOL = 6, 4, 30, 1e-6
BUILD_TIMED_EVERY = 4   # timed solves per one whose build records its sweep events
METRIC = "preconditioned FGMRES solves/s at 1e-6; sweep GB/s vs HBM peak; p50/p99 latency"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each
# kernel from one ncu --set full capture of that kernel on this workload (same
# kernel code; set an entry to None when its kernel changes until it is
# captured again)
PROFILED_TRAFFIC = {
    "spmv_f64": 295.448832e6 + 15.170560e6,          # k_spmv<1>
    "build_sweeps_f32": 1.392420e9 + 531.461376e6,    # k_build_blocks_async<float, 1, 64>,
                                                       # 6 sweeps, strided 128-block tickets
    "lower_sweeps_f32": 131.777024e6 + 6.098432e6,     # k_tri_staged<0, 0, 0, float>, 3 sweeps
    "upper_sweeps_f32": 81.267456e6 + 1.445632e6,      # k_tri_staged<1, 1, 0, float>, 3 sweeps
}


def max_over_ranks(torch, value, device):
    """Largest value over all ranks (the job's wall time is the slowest rank's)."""
    if not torch.distributed.is_available() or not torch.distributed.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, max_ms):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return world * units_per_rank / (max_ms * 1e-3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def begin(self):
        self.t0 = datetime.datetime.now()

    def end(self):
        self.t1 = datetime.datetime.now()

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
                rows.append((ts, float(f[1]), float(f[2]),
                             {nm for nm, v in zip(names, f[4:8]) if v.lower() == "active"}))
            except ValueError:
                continue
        if not rows:
            return None
        # the samples taken inside [begin, end]; a region shorter than the
        # sampling interval keeps the sample nearest to its middle
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 <= r[0] <= self.t1]
        if not inside:
            mid = self.t0 + (self.t1 - self.t0) / 2 if self.t0 and self.t1 else rows[0][0]
            inside = [min(rows, key=lambda r: abs((r[0] - mid).total_seconds()))]
        reasons = set().union(*(r[3] for r in inside))
        out = {"sm_mhz": statistics.median(r[1] for r in inside),
               "sm_max_mhz": max(r[2] for r in inside), "reasons": sorted(reasons),
               "samples": len(inside), "samples_total": len(rows)}
        if self.t0 and self.t1:
            out["region_s"] = round((self.t1 - self.t0).total_seconds(), 3)
        return out


def _system():
    import abilu_inputs as gen
    return gen.workload(WORKLOAD)


# ------------------------------------------------------------------ oracle arm

def oracle_solve(s, max_iters=2500):
    import oracle
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, BUILD_SWEEPS)
    x, r = oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, s.b, APPLY_SWEEPS, APPLY_SWEEPS,
                         restart=RESTART, max_iters=max_iters, rtol=RTOL)
    return r


def oracle_solution(s, max_iters=2500):
    """The FP64 oracle's solution x and result of the workload's solve."""
    import oracle
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, BUILD_SWEEPS)
    return oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, s.b, APPLY_SWEEPS, APPLY_SWEEPS,
                         restart=RESTART, max_iters=max_iters, rtol=RTOL)


def host_cpu():
    """nproc and the CPU model of this host (lscpu's model name, else
    /proc/cpuinfo's)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown",
            "machine": os.uname().machine}


def oracle_kernel_ms(s, reps=2):
    """The oracle's time (one host core, FP64) for one synchronous build sweep,
    one lower sweep, one upper sweep and one SpMV of workload s, best of reps."""
    import numpy as np
    import oracle
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    r = np.random.default_rng(1).standard_normal((s.n, 4))
    y0 = np.zeros_like(r)

    def best(fn):
        t = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            t.append(time.perf_counter() - t0)
        return round(1e3 * min(t), 2)
    return {"build_sweep": best(lambda: oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, X, D)),
            "lower_sweep": best(lambda: oracle.lower_sweep(s.rowptr, s.colind, X, r, y0)),
            "upper_sweep": best(lambda: oracle.upper_sweep(s.rowptr, s.colind, X, D, r, y0)),
            "spmv": best(lambda: oracle.spmv(s.rowptr, s.colind, s.vals, r))}


def cpu_baseline(s, budget_s=12.0, viscous=None):
    """Full oracle solves (FP64, one host thread) until ~budget_s of CPU time;
    the oracle's per-kernel times on this workload (and on `viscous`)."""
    t0 = time.perf_counter()
    n = 0
    while True:
        x_or, r = oracle_solution(s)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 5:
            break
    out = {"value": n / el, "unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} full FP64 oracle solves of the 512x512 workload (sync build "
                     f"{BUILD_SWEEPS} sweeps, {APPLY_SWEEPS}+{APPLY_SWEEPS} apply sweeps, "
                     f"FGMRES({RESTART}) to {RTOL:g}, {r.iters} iterations each) in {el:.1f} s "
                     f"on one host core",
           **host_cpu(),
           "oracle_kernel_ms": {WORKLOAD: oracle_kernel_ms(s)}}
    if viscous is not None:
        out["oracle_kernel_ms"][viscous.name] = oracle_kernel_ms(viscous)
    return out, x_or, r


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    s = _system()
    for _ in range(args.warmup):
        oracle_solve(s)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle_solve(s)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": s.n, "blocks": s.nnzb,
                       "build_sweeps": BUILD_SWEEPS, "apply_sweeps": APPLY_SWEEPS,
                       "restart": RESTART, "rtol": RTOL, "iters": r.iters},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step one full FP64 oracle solve ({r.iters} "
                                       "FGMRES iterations) on one host core"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# -------------------------------------------------------------------- GPU arm

def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def kernel_rooflines(torch, ab, pat, A, fac, s, peak, mode="async"):
    """Average duration of the hot kernels, each isolated as the difference of
    two public calls timed with CUDA events on the launching stream
    (back-to-back calls after warm-up), and achieved GB/s from the algorithmic
    bytes of one launch (the per-kernel formulas are written out below).  FP32
    factors."""
    N, nnzb = s.n, s.nnzb
    E = (nnzb - N) // 2
    f, v = 4, 4   # FP32 factors, FP32 apply vectors
    c = pat.counts()
    nw, npairs = c["nwork"], c["npairs"]
    x = torch.randn(N, 4, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    reps = 40

    def avg_us(fn):
        for _ in range(5):
            fn()
        e0, e1 = _events(torch, 2)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e3

    out = {}
    t = avg_us(lambda: ab.bsr_spmv(pat, A, x, y))
    out["spmv_f64"] = {"us": t, "bytes": nnzb * (128 + 4) + 4 * (N + 1) + 2 * 32 * N,
                       "sweeps": 1}
    # build: prepare pass + sweeps; the sweeps are the difference to 0 sweeps.
    # One sweep's unique bytes over the work list: the 32-byte records, FP32 A
    # rows, the pair list (counted whole, though the first two pairs of a block
    # sit in its record), the pairs' L and U rows, Dinv read and written, L written
    sweep_b = (nw * 32 + nw * 16 * f + npairs * 8 + 2 * npairs * 16 * f
               + 2 * N * 16 * f + c["nl"] * 16 * f)
    nb = BUILD_SWEEPS
    t0 = avg_us(lambda: fac.build(A, 0, mode, init="previous"))
    tb = avg_us(lambda: fac.build(A, nb, mode, init="previous"))
    if mode == "async":   # one persistent launch runs all sweeps
        out["build_sweeps_f32"] = {"us": tb - t0, "bytes": nb * sweep_b, "sweeps": nb}
    else:
        out["build_sweep_f32"] = {"us": (tb - t0) / nb, "bytes": sweep_b, "sweeps": 1}
    # prepare (warm start): A read once, FP32 copy of the work blocks, constant
    # U blocks (into both buffers for sync builds), index arrays
    ncu_ = c["nu"] - (nw - c["nl"] - N)
    # plus, after the sweeps, the Dinv-scaled upper blocks (FP32 factors): U and
    # Dinv read, Us written
    out["build_prepare_f32"] = {"us": t0, "bytes": nnzb * 128 + 4 * (nnzb + 1) + 16 * (N + 1)
                                + nw * 16 * f + (2 if mode == "sync" else 1) * ncu_ * 16 * f
                                + 2 * c["nu"] * 16 * f + N * 16 * f + 4 * (N + 1),
                                "sweeps": 1}
    # a sweep reads its factor blocks and column indices, the right-hand side and
    # the gathered neighbour values, and writes its vector; the upper sweeps run
    # on Us = Dinv U with right-hand side Dinv y, so no Dinv read
    bl = E * (16 * f + 4) + 4 * (N + 1) + 3 * N * 4 * v
    bu = E * (16 * f + 4) + 4 * (N + 1) + 3 * N * 4 * v
    # both modes take the first update of each factor without a sweep (y = r,
    # x^1 = Dinv y); the sweeps are the difference to one update per factor
    na = APPLY_SWEEPS
    t11 = avg_us(lambda: fac.apply(x, z, 1, 1, mode))
    tl = avg_us(lambda: fac.apply(x, z, na, 1, mode)) - t11
    tu = avg_us(lambda: fac.apply(x, z, 1, na, mode)) - t11
    if mode == "async":   # one in-place launch runs the na - 1 sweeps
        out["lower_sweeps_f32"] = {"us": tl, "bytes": (na - 1) * bl, "sweeps": na - 1}
        out["upper_sweeps_f32"] = {"us": tu, "bytes": (na - 1) * bu, "sweeps": na - 1}
    else:
        out["lower_sweep_f32"] = {"us": tl / (na - 1), "bytes": bl, "sweeps": 1}
        out["upper_sweep_f32"] = {"us": tu / (na - 1), "bytes": bu, "sweeps": 1}
    for k in out.values():
        k["GBs"] = k["bytes"] / (k["us"] * 1e-6) / 1e9
        k["frac"] = k["GBs"] / peak
    return out


def run_kernels_only(args):
    """Per-kernel timings only (the target of the ncu captures)."""
    import torch
    import paper_1912_00539_gb300 as ab
    peak, _ = _peaks()
    s = _system()
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    A = torch.from_numpy(s.vals).cuda()
    out = {}
    for mode in ("async", "sync"):
        fk = ab.Factors(pat, "f32")
        fk.build(A, BUILD_SWEEPS, mode)
        kern = kernel_rooflines(torch, ab, pat, A, fk, s, peak, mode)
        out[mode] = {k: {kk: round(vv, 3) for kk, vv in v.items()} for k, v in kern.items()}
    print(json.dumps(out))
    return 0


def run_profile_solves(args):
    """Warm-up plus --profile-solves solves of the timed step and nothing else:
    the command the ncu launch list is taken on."""
    import torch
    import paper_1912_00539_gb300 as ab
    s = _system()
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    A = torch.from_numpy(s.vals).cuda()
    b = torch.from_numpy(s.b).cuda()
    x = torch.zeros_like(b)
    fac = ab.Factors(pat, args.dtype)
    for _ in range(args.warmup + args.profile_solves):
        r = ab.fgmres_solve(pat, A, fac, b, x, restart=RESTART, rtol=RTOL,
                            build_sweeps=BUILD_SWEEPS, apply_sweeps_lower=APPLY_SWEEPS,
                            apply_sweeps_upper=APPLY_SWEEPS, mode=args.mode, raise_on_noconv=True,
                            zero_guess=True)
    torch.cuda.synchronize()
    print(json.dumps({"solves": args.warmup + args.profile_solves, "iters": r.iters,
                      "rel_resid_true": r.rel_resid_true}))
    return 0


def run_profile_batch(args):
    """Warm-up plus --profile-batch solves of the 64-system batch with fixed
    settings (4 build, 3+3 apply sweeps, sync; no autotuning): the command the
    batch's launch list is taken on."""
    import torch
    import abilu_inputs as gen
    import paper_1912_00539_gb300 as ab
    systems = gen.batch_systems(64)
    dev = [(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda(),
            torch.from_numpy(s.vals).cuda(), torch.from_numpy(s.b).cuda()) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in dev], dtype="f32")
    for k, d in enumerate(dev):
        batch.set_system(k, d[2], d[3])
    for _ in range(args.warmup + args.profile_batch):
        res = batch.solve(restart=RESTART, rtol=RTOL, build_sweeps=4, apply_sweeps_lower=3,
                          apply_sweeps_upper=3, mode="sync")
    torch.cuda.synchronize()
    print(json.dumps({"solves": args.warmup + args.profile_batch,
                      "cells": sum(s.n for s in systems), "iters_max": max(r.iters for r in res)}))
    return 0


def run_profile_mg(args):
    """Warm-up plus --profile-mg FGMRES solves preconditioned by the V-cycle
    (512x512 workload, FP32 factors, synchronous 2+2 smoothing, 6 build sweeps
    per level): the command the multigrid launch list is taken on."""
    import torch
    import paper_1912_00539_gb300 as ab
    s = _system()
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    A = torch.from_numpy(s.vals).cuda()
    b = torch.from_numpy(s.b).cuda()
    x = torch.zeros_like(b)
    mg = ab.Multigrid(pat, A, factor_dtype="f32", build_sweeps=BUILD_SWEEPS, apply_sweeps_lower=2,
                      apply_sweeps_upper=2, mode="sync")
    for _ in range(args.warmup + args.profile_mg):
        r = ab.fgmres_solve_mg(mg, A, b, x, restart=RESTART, rtol=RTOL, zero_guess=True,
                               raise_on_noconv=True)
    torch.cuda.synchronize()
    print(json.dumps({"solves": args.warmup + args.profile_mg, "levels": mg.cells,
                      "iters": r.iters, "rel_resid_true": r.rel_resid_true}))
    return 0


def run_batched(args, nsys=64, steps=3):
    """64 uneven systems (2k-200k cells, aspect 1/8-8, CFL 10-1e4), FP32
    factors, FGMRES(30) to 1e-6: the batch solved in the same launches vs the
    same systems solved one after another through the single-system API."""
    import torch
    import abilu_inputs as gen
    import paper_1912_00539_gb300 as ab
    t0 = time.perf_counter()
    systems = gen.batch_systems(nsys)
    tgen = time.perf_counter() - t0
    dev = [(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda(),
            torch.from_numpy(s.vals).cuda(), torch.from_numpy(s.b).cuda()) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in dev], dtype="f32")
    for k, d in enumerate(dev):
        batch.set_system(k, d[2], d[3])
    cells = sum(s.n for s in systems)
    from paper_1912_00539_gb300 import autotune
    t0 = time.perf_counter()
    cfls = [s.cfl for s in systems]
    choice = autotune.tune_batch(batch, cells, restart=RESTART, rtol=RTOL,
                                 cfl_range=(min(cfls), max(cfls)))
    ttune = time.perf_counter() - t0
    opts = dict(restart=RESTART, rtol=RTOL, build_sweeps=choice.build_sweeps,
                apply_sweeps_lower=choice.apply_sweeps, apply_sweeps_upper=choice.apply_sweeps,
                mode=choice.mode)
    res = batch.solve(**opts)
    torch.cuda.synchronize()
    e0, e1 = _events(torch, 2)
    e0.record()
    for _ in range(steps):
        res = batch.solve(**opts)
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / steps
    pats = [ab.Pattern(d[0], d[1]) for d in dev]
    facs = [ab.Factors(p, "f32") for p in pats]
    xs = [torch.zeros_like(d[3]) for d in dev]

    def one_by_one():
        out = []
        for d, p, f, x in zip(dev, pats, facs, xs):
            x.zero_()
            out.append(ab.fgmres_solve(p, d[2], f, d[3], x, **opts))
        return out

    r1 = one_by_one()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        r1 = one_by_one()
    e1.record()
    torch.cuda.synchronize()
    t1 = e0.elapsed_time(e1) / steps
    return {"workload": f"batch of {nsys} systems, {cells} cells", "cells": cells,
            "autotuned": {"build_sweeps": choice.build_sweeps, "apply_sweeps": choice.apply_sweeps,
                          "build_chunk": choice.build_chunk,
                          "key": autotune.cfl_bucket(min(cfls), max(cfls)),
                          "mode": choice.mode, "tuning_s": round(ttune, 1)},
            "batch_ms": round(tb, 3), "batch_systems_per_s": round(nsys / (tb * 1e-3), 1),
            "one_by_one_ms": round(t1, 3), "one_by_one_systems_per_s": round(nsys / (t1 * 1e-3), 1),
            "converged": sum(r.converged for r in res), "iters_max": max(r.iters for r in res),
            "iters_min": min(r.iters for r in res),
            "iters_one_by_one_max": max(r.iters for r in r1), "generation_s": round(tgen, 1)}


def _r(v):
    """Round for the report without zeroing small magnitudes."""
    return float(f"{v:.4g}") if isinstance(v, float) else v


def _rd(d):
    return {k: ({kk: _r(vv) for kk, vv in v.items()} if isinstance(v, dict) else _r(v))
            for k, v in d.items()}


def run_serving(args, n_requests=48, rates=(0.25, 0.5, 1.0, 1.5), reps=3):
    """Poisson stream of requests (4k-1M cells log-uniform, 5 value updates
    each, CFL x4 per update), FP32 factors, served by continuous batching (every
    step one update of every admitted request in shared launches, warm-started
    factors, admission by room in an arena sized to the HBM budget); against
    plain FP64 ABILU (synchronous sweeps) solving the requests one at a time on
    the same GPU.  Capacity = solves/s with every request queued at t = 0; the
    arrival rates are fractions of it.  Every configuration runs `reps` times
    after one untimed run and reports its median run (by solves/s), with the
    solves/s of all timed runs in the order they ran:
    the host's own load moves single runs (one run of the 20-request stream at
    the 1.0x rate stalled for 0.35 s on a loaded host)."""
    import torch
    import abilu_inputs as gen
    from paper_1912_00539_gb300 import serving
    t0 = time.perf_counter()
    stream = gen.serving_stream(rate_hz=1.0, n_requests=n_requests, seed=5)
    tgen = time.perf_counter() - t0
    # every update's values and right-hand side in pinned host memory, once
    unit = [serving.Request(r.rid, r.arrival, r.system.rowptr, r.system.colind,
                            [(torch.from_numpy(v).pin_memory(), torch.from_numpy(b).pin_memory())
                             for v, b, _ in r.updates]) for r in stream]
    del stream
    n_upd = sum(len(r.updates) for r in unit)

    def at_rate(rate):
        return [serving.Request(r.rid, r.arrival / rate, r.rowptr, r.colind, r.updates)
                for r in unit]

    budget = 0.25 * torch.cuda.get_device_properties(0).total_memory
    cfg = dict(build_sweeps=args.batch_build_sweeps, apply_sweeps=args.batch_apply_sweeps)
    def median_run(run):
        # one untimed run of the configuration first: in the 20-request stream
        # the first of a configuration's runs, which follows host-only work
        # that leaves the GPU idle, was the slowest in every configuration
        # (e.g. 636 against 1,045 and 1,211 solves/s)
        run()
        runs = [serving.summarize(*run()) for _ in range(reps)]   # in the order they ran
        med = dict(sorted(runs, key=lambda r: r["solves_per_s"])[len(runs) // 2])
        med["runs_solves_per_s"] = [round(r["solves_per_s"], 1) for r in runs]
        return med

    srv = serving.Server(budget, dtype="f32", mode=args.mode, **cfg)
    cap = median_run(lambda: srv.run(at_rate(1e9)))   # capacity: all queued at t = 0
    req_rate = cap["requests"] / cap["wall_s"]
    out = {"workload": f"{n_requests} requests, 4k-1M cells (log-uniform), 5 updates each",
           "cells": int(sum(r.n for r in unit)), "updates": n_upd, "generation_s": round(tgen, 1),
           "arena": {"cells": srv.cells, "blocks": srv.blocks, "bytes": srv.arena_bytes,
                     "budget_bytes": budget},
           "f32_capacity": _rd(cap)}
    for frac in rates:
        out[f"f32_rate_{frac}x"] = _rd(median_run(lambda: srv.run(at_rate(frac * req_rate))))
    srv.close()
    # the baseline: plain FP64 ABILU, one request at a time (all queued at t = 0
    # for its capacity, and at the 1.0x arrival rate)
    out["f64_one_at_a_time_capacity"] = _rd(median_run(
        lambda: serving.serve_one_at_a_time(at_rate(1e9), dtype="f64", mode="sync", **cfg)))
    out["f64_one_at_a_time_rate_1.0x"] = _rd(median_run(
        lambda: serving.serve_one_at_a_time(at_rate(1.0 * req_rate), dtype="f64", mode="sync",
                                            **cfg)))
    out["f32_serving_over_f64_one_at_a_time"] = round(
        cap["solves_per_s"] / out["f64_one_at_a_time_capacity"]["solves_per_s"], 3)
    return out


def viscous_rcm_vs_line(steps=5):
    """The viscous-like 1024x256 workload in its two orderings (RCM, whole
    wall-normal lines): FP32 factors, asynchronous, 8 build and 6+6 apply
    sweeps, FGMRES(50) to 1e-6, against the FP64 oracle's iterations and
    solution."""
    import numpy as np
    import torch
    import abilu_inputs as gen
    import oracle
    import paper_1912_00539_gb300 as ab
    out = {}
    for order in ("rcm", "line"):
        name = f"viscous_1024x256_{order}"
        s = gen.workload(name)
        st = gen.SOLVER_SETTINGS[name]
        pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
        A = torch.from_numpy(s.vals).cuda()
        b = torch.from_numpy(s.b).cuda()
        fac = ab.Factors(pat, "f32")
        x = torch.zeros_like(b)

        def solve():
            return ab.fgmres_solve(pat, A, fac, b, x, restart=st["restart"], rtol=st["rtol"],
                                   build_sweeps=st["build_sweeps"],
                                   apply_sweeps_lower=st["apply_sweeps"],
                                   apply_sweeps_upper=st["apply_sweeps"], mode="async",
                                   zero_guess=True)
        r = solve()
        torch.cuda.synchronize()
        e0, e1 = _events(torch, 2)
        e0.record()
        for _ in range(steps):
            r = solve()
        e1.record()
        torch.cuda.synchronize()
        Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, st["build_sweeps"])
        xo, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, st["apply_sweeps"],
                               st["apply_sweeps"], restart=st["restart"], rtol=st["rtol"])
        xn = x.cpu().numpy()
        out[order] = {"solves_per_s": round(steps / (e0.elapsed_time(e1) * 1e-3), 1),
                      "iters": r.iters, "oracle_f64_iters": ro.iters,
                      "rel_resid_true": _r(r.rel_resid_true),
                      "err_vs_oracle": _r(float(np.linalg.norm(xn - xo) / np.linalg.norm(xo)))}
    return out


def run_continuation(args):
    """Pseudo-time continuation (Sec. 2) of a steady model problem
    r(w) = A w + 0.5 w|w| - f on the 512x512 grid's block pattern, from w = 0
    to a 1e-6 drop of the energy residual: CFL ramp of Eq. (cfl) from 10 to
    1e4, each step FGMRES(30) to a 0.1 drop (at most 60 iterations) with ABILU
    (1 build sweep, 3+3 apply sweeps) warm-started from the previous step's
    factors, against the same march with FP64 factors and synchronous sweeps."""
    import torch
    import abilu_inputs as gen
    import paper_1912_00539_gb300 as ab
    from paper_1912_00539_gb300.continuation import PseudoTimeSolver, SemilinearProblem
    case = gen.semilinear_case(512, 512)
    s = case.system
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    A = torch.from_numpy(s.vals).cuda()
    ws = torch.from_numpy(case.w_star).cuda()
    f = torch.empty_like(ws)
    ab.bsr_spmv(pat, A, ws, f)                      # f = A w* + kappa w*|w*|
    f.addcmul_(ws, ws.abs(), value=case.kappa)
    prob = SemilinearProblem(pat, A, f, case.kappa)
    scale = torch.from_numpy(case.shift_scale).cuda()
    out = {"workload": f"semilinear model problem on the 512x512 grid ({s.n} cells), "
                       "w = 0 to a 1e-6 energy-residual drop"}
    for dt, md in (("f32", "async"), ("f64", "sync")):
        drv = PseudoTimeSolver(pat, prob.residual, prob.jacobian, scale, dtype=dt, mode=md)
        w = torch.zeros_like(ws)
        drv.run(w, rel_tol=1e-6, max_steps=3)      # warm-up (allocations, occupancy lookups)
        w.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        log = drv.run(w, rel_tol=1e-6, max_steps=500)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        err = float(torch.linalg.vector_norm(w - ws) / torch.linalg.vector_norm(ws))
        out[f"{dt}_{md}"] = {
            "steps": len(log), "linear_iters": sum(st.lin_iters for st in log),
            "wall_s": round(wall, 4), "ms_per_step": round(wall * 1e3 / len(log), 3),
            "final_cfl": round(log[-1].cfl, 1),
            "energy_residual_drop": _r(log[-1].energy / float(torch.linalg.vector_norm(f[:, 3]))),
            "rel_error_vs_manufactured": _r(err)}
    return out


def run_scalar_vs_block(args):
    """The paper's central comparison (Sec. 6): asynchronous block ILU(0)
    against the scalar (Chow-Patel) ILU(0) on the same matrices, FP64 factors,
    synchronous and asynchronous sweeps, FGMRES to 1e-6 (at most 500
    iterations): iterations, convergence and solves/s."""
    import numpy as np
    import torch
    import abilu_inputs as gen
    import paper_1912_00539_gb300 as ab
    cases = [("inviscid_512x512", gen.workload("inviscid_512x512"),
              gen.SOLVER_SETTINGS["inviscid_512x512"]),
             ("viscous_1024x256_rcm", gen.workload("viscous_1024x256_rcm"),
              gen.SOLVER_SETTINGS["viscous_1024x256_rcm"]),
             ("viscous_1024x256_line", gen.workload("viscous_1024x256_line"),
              gen.SOLVER_SETTINGS["viscous_1024x256_line"])]
    out = {}
    for name, s, st in cases:
        pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
        A = torch.from_numpy(s.vals).cuda()
        b = torch.from_numpy(np.ascontiguousarray(s.b)).cuda()
        row = {}
        for variant in ("block", "scalar"):
            for md in ("sync", "async"):
                fac = ab.Factors(pat, "f64", scalar=variant == "scalar")
                x = torch.zeros_like(b)

                def solve():
                    x.zero_()
                    return ab.fgmres_solve(pat, A, fac, b, x, restart=st["restart"],
                                           max_iters=500, rtol=st["rtol"],
                                           build_sweeps=st["build_sweeps"],
                                           apply_sweeps_lower=st["apply_sweeps"],
                                           apply_sweeps_upper=st["apply_sweeps"], mode=md)
                r = solve()
                torch.cuda.synchronize()
                e0, e1 = _events(torch, 2)
                e0.record()
                for _ in range(3):
                    r = solve()
                e1.record()
                torch.cuda.synchronize()
                row[f"{variant}_{md}"] = {"iters": r.iters, "converged": r.converged,
                                          "rel_resid_true": _r(r.rel_resid_true),
                                          "solves_per_s": round(3 / (e0.elapsed_time(e1) * 1e-3), 1)}
        out[name] = row
    return out


def run_viscous(args):
    """Viscous-like anisotropic grid (1024x256, CFL 1e4, wall-normal coupling
    x100): RCM vs wall-normal line ordering, FP32 factors, 8 build and 6+6
    apply sweeps, FGMRES(50) to 1e-6; iterations against the FP64 oracle."""
    import numpy as np
    import torch
    import abilu_inputs as gen
    import oracle
    import paper_1912_00539_gb300 as ab
    out = {}
    for order in ("rcm", "line"):
        name = f"viscous_1024x256_{order}"
        s = gen.workload(name)
        st = gen.SOLVER_SETTINGS[name]
        pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
        A = torch.from_numpy(s.vals).cuda()
        b = torch.from_numpy(s.b).cuda()
        Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, st["build_sweeps"])
        _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, st["apply_sweeps"],
                              st["apply_sweeps"], restart=st["restart"], rtol=st["rtol"])
        row = {"oracle_f64_iters": ro.iters}
        for dt, md in (("f32", "sync"), ("f32", "async"), ("f64", "sync")):
            fac = ab.Factors(pat, dt)
            x = torch.zeros_like(b)

            def solve():
                x.zero_()
                return ab.fgmres_solve(pat, A, fac, b, x, restart=st["restart"], rtol=st["rtol"],
                                       build_sweeps=st["build_sweeps"],
                                       apply_sweeps_lower=st["apply_sweeps"],
                                       apply_sweeps_upper=st["apply_sweeps"], mode=md)
            r = solve()
            torch.cuda.synchronize()
            e0, e1 = _events(torch, 2)
            e0.record()
            for _ in range(5):
                r = solve()
            e1.record()
            torch.cuda.synchronize()
            row[f"{dt}_{md}"] = {"iters": r.iters, "rel_resid_true": r.rel_resid_true,
                                 "solves_per_s": round(5 / (e0.elapsed_time(e1) * 1e-3), 1)}
        out[order] = row
    # the library's orderings of the same grid (from its natural numbering):
    # RCM, one-way dissection, lines found from the block norms, and the
    # hybrid line-RCM / line-1WD orderings of the graph of lines and cells
    s0 = gen.make_system(1024, 256, 301, 302, 303, 1.0e4, order="natural", wall_normal_scale=100.0)
    st = gen.SOLVER_SETTINGS["viscous_1024x256_rcm"]
    lib = {}
    for kind in ("rcm", "1wd", "line", "line-rcm", "line-1wd"):
        t0 = time.perf_counter()
        perm, line_of = ab.order(s0.rowptr, s0.colind, kind, vals=s0.vals, line_threshold=10.0)
        t_order = time.perf_counter() - t0
        ro, co, src = ab.permute_pattern(s0.rowptr, s0.colind, perm)
        pat = ab.Pattern(torch.from_numpy(ro).cuda(), torch.from_numpy(co).cuda())
        A0 = torch.from_numpy(s0.vals).cuda()
        A = torch.empty_like(A0)
        ab.gather_blocks(torch.from_numpy(src).cuda(), A0, A)
        b = torch.from_numpy(np.ascontiguousarray(s0.b[perm])).cuda()
        row = {"lines": int(line_of.max() + 1), "order_s": round(t_order, 3)}
        for dt, md in (("f32", "sync"), ("f32", "async")):
            fac = ab.Factors(pat, dt)
            x = torch.zeros_like(b)

            def solve():
                x.zero_()
                return ab.fgmres_solve(pat, A, fac, b, x, restart=st["restart"], rtol=st["rtol"],
                                       build_sweeps=st["build_sweeps"],
                                       apply_sweeps_lower=st["apply_sweeps"],
                                       apply_sweeps_upper=st["apply_sweeps"], mode=md)
            r = solve()
            torch.cuda.synchronize()
            e0, e1 = _events(torch, 2)
            e0.record()
            for _ in range(5):
                r = solve()
            e1.record()
            torch.cuda.synchronize()
            row[f"{dt}_{md}"] = {"iters": r.iters, "rel_resid_true": _r(r.rel_resid_true),
                                 "solves_per_s": round(5 / (e0.elapsed_time(e1) * 1e-3), 1)}
        lib[kind] = row
    out["library_orderings"] = lib
    return out


def run_multigrid(args):
    """Block ILU sweeps as a multigrid smoother (the paper's future work):
    FGMRES preconditioned by an aggregation V-cycle against the single-level
    block ILU preconditioner on the 512x512 and viscous-like grids: levels,
    iterations (with the FP64 oracle's), solves/s, the time of one V-cycle,
    and the convergence factor of the V-cycle used as a stationary iteration
    x += V(b - A x) with synchronous and asynchronous smoothing sweeps."""
    import numpy as np
    import torch
    import abilu_inputs as gen
    import oracle
    import paper_1912_00539_gb300 as ab
    out = {}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = _events(torch, 2)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / reps

    for name in ("inviscid_512x512", "viscous_1024x256_rcm"):
        s = gen.workload(name)
        st = gen.SOLVER_SETTINGS[name]
        pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
        A = torch.from_numpy(s.vals).cuda()
        b = torch.from_numpy(np.ascontiguousarray(s.b)).cuda()
        x = torch.zeros_like(b)
        row = {}
        fac = ab.Factors(pat, "f32")

        def plain():
            x.zero_()
            return ab.fgmres_solve(pat, A, fac, b, x, restart=st["restart"], rtol=st["rtol"],
                                   build_sweeps=st["build_sweeps"],
                                   apply_sweeps_lower=st["apply_sweeps"],
                                   apply_sweeps_upper=st["apply_sweeps"], mode="async")
        r, ms = timed(plain, 5)
        row["abilu_f32_async"] = {"iters": r.iters, "rel_resid_true": _r(r.rel_resid_true),
                                  "ms": round(ms, 3), "solves_per_s": round(1e3 / ms, 1)}
        nb = st["build_sweeps"]
        lv = oracle.mg_hierarchy(s.rowptr, s.colind, s.vals, build_sweeps=nb)
        _, ro = oracle.fgmres_mg(lv, s.b, 2, 2, pre=1, post=1, coarse=2, restart=st["restart"],
                                 rtol=st["rtol"], max_iters=300)
        row["oracle_mg_f64_2+2_iters"] = ro.iters
        for md, sw, mc in (("sync", 1, 512), ("sync", 2, 512), ("async", 1, 512),
                           ("async", 2, 512), ("sync", 2, 8192), ("async", 2, 8192),
                           ("sync", 2, 65536), ("async", 2, 65536)):
            mg = ab.Multigrid(pat, A, factor_dtype="f32", build_sweeps=nb,
                              apply_sweeps_lower=sw, apply_sweeps_upper=sw, mode=md,
                              min_coarse=mc)

            def solve():
                x.zero_()
                return ab.fgmres_solve_mg(mg, A, b, x, restart=st["restart"], rtol=st["rtol"],
                                          max_iters=300)
            r, ms = timed(solve, 5)
            rr = torch.empty_like(b)
            z = torch.empty_like(b)
            _, ms_cycle = timed(lambda: mg.apply(b, z), 20)
            # V-cycle as a stationary iteration: residual reduction per cycle
            x.zero_()
            bnorm = float(torch.linalg.vector_norm(b))
            for _ in range(10):
                rr.copy_(b)
                ab.bsr_spmv(pat, A, x, rr, alpha=-1.0, beta=1.0)
                mg.apply(rr, z)
                x.add_(z)
            rr.copy_(b)
            ab.bsr_spmv(pat, A, x, rr, alpha=-1.0, beta=1.0)
            rho = (float(torch.linalg.vector_norm(rr)) / bnorm) ** 0.1
            row[f"mg_f32_{md}_{sw}+{sw}_min{mc}"] = {
                "levels": mg.nlevels, "cells": mg.cells, "iters": r.iters,
                "rel_resid_true": _r(r.rel_resid_true), "ms": round(ms, 3),
                "solves_per_s": round(1e3 / ms, 1), "vcycle_ms": round(ms_cycle, 3),
                "stationary_factor": round(rho, 4)}
        # the same stationary iteration with the single-level smoother
        for md in ("sync", "async"):
            mg1 = ab.Multigrid(pat, A, max_levels=1, factor_dtype="f32", build_sweeps=nb,
                               apply_sweeps_lower=2, apply_sweeps_upper=2, coarse_smooth=1, mode=md)
            mg1.setup(A)
            x.zero_()
            rr = torch.empty_like(b)
            z = torch.empty_like(b)
            for _ in range(10):
                rr.copy_(b)
                ab.bsr_spmv(pat, A, x, rr, alpha=-1.0, beta=1.0)
                mg1.apply(rr, z)
                x.add_(z)
            rr.copy_(b)
            ab.bsr_spmv(pat, A, x, rr, alpha=-1.0, beta=1.0)
            row[f"smoother_only_f32_{md}_2+2_stationary_factor"] = round(
                (float(torch.linalg.vector_norm(rr)) / float(torch.linalg.vector_norm(b))) ** 0.1, 4)
        out[name] = row
    return out


def run_parilut(args):
    """Threshold block ILU (fill of L U added, largest blocks kept, synchronous
    sweeps; FP64 factors) against block ILU(0) on the 512x512 and viscous-like
    grids: set-up time, blocks, FGMRES iterations and solve time with the
    factors reused (the threshold factorisation is a set-up that several
    right-hand sides or pseudo-time steps share), with the oracle's counts."""
    import numpy as np
    import torch
    import abilu_inputs as gen
    import oracle
    import paper_1912_00539_gb300 as ab
    out = {}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = _events(torch, 2)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / reps

    for name in ("inviscid_512x512", "viscous_1024x256_rcm"):
        s = gen.workload(name)
        st = gen.SOLVER_SETTINGS[name]
        na = st["apply_sweeps"]
        pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
        A = torch.from_numpy(s.vals).cuda()
        b = torch.from_numpy(np.ascontiguousarray(s.b)).cuda()
        x = torch.zeros_like(b)
        row = {"A_blocks": int(s.nnzb)}
        for dt in ("f64", "f32"):
            fac = ab.Factors(pat, dt)
            fac.build(A, st["build_sweeps"], mode="async")

            def solve0():
                x.zero_()
                return ab.fgmres_solve(pat, A, fac, b, x, restart=st["restart"], rtol=st["rtol"],
                                       apply_sweeps_lower=na, apply_sweeps_upper=na, mode="async",
                                       build=False, max_iters=300)
            r, ms = timed(solve0, 5)
            row[f"ilu0_{dt}_async"] = {"iters": r.iters, "solve_ms": round(ms, 3)}
        for fill, fdt in ((1.5, "f64"), (2.0, "f64"), (1.5, "f32"), (2.0, "f32")):
            t0 = time.perf_counter()
            fpat, ffac = ab.parilut(pat, A, fill=fill, iters=3, sweeps=2, dtype=fdt)
            t_setup = time.perf_counter() - t0
            _, t_setup2 = timed(lambda: ab.parilut(pat, A, fill=fill, iters=3, sweeps=2, dtype=fdt),
                                2)
            rec = {"blocks": fpat.nnzb, "setup_ms": round(t_setup2, 2),
                   "first_setup_ms": round(t_setup * 1e3, 1)}
            for md in ("sync", "async"):
                def solve():
                    x.zero_()
                    return ab.fgmres_solve(pat, A, ffac, b, x, restart=st["restart"],
                                           rtol=st["rtol"], apply_sweeps_lower=na,
                                           apply_sweeps_upper=na, mode=md, build=False,
                                           max_iters=300)
                r, ms = timed(solve, 5)
                rec[f"{md}_iters"] = r.iters
                rec[f"{md}_solve_ms"] = round(ms, 3)
                rec[f"{md}_rel_resid_true"] = _r(r.rel_resid_true)
            if fdt == "f64":
                rp, ci, Xo, Do = oracle.parilut(s.rowptr, s.colind, s.vals, fill=fill, iters=3,
                                                sweeps=2)
                _, ro = oracle.fgmres_ilu_pattern(s.rowptr, s.colind, s.vals, rp, ci, Xo, Do, s.b,
                                                  na, na, restart=st["restart"], max_iters=300)
                rec["oracle_blocks"] = int(len(ci))
                rec["oracle_iters"] = ro.iters
            row[f"threshold_fill{fill}_{fdt}"] = rec
        out[name] = row
    return out


def run_gpu(args):
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1912_00539_gb300 as ab
    peak, peak_kind = _peaks()
    s = _system()
    dev = torch.device("cuda", local)
    rowptr = torch.from_numpy(s.rowptr).to(dev)
    colind = torch.from_numpy(s.colind).to(dev)
    A = torch.from_numpy(s.vals).to(dev)
    b = torch.from_numpy(s.b).to(dev)
    x = torch.zeros_like(b)
    pat = ab.Pattern(rowptr, colind)
    fac = ab.Factors(pat, args.dtype)
    stream = torch.cuda.current_stream()

    def solve():
        return ab.fgmres_solve(pat, A, fac, b, x, restart=RESTART, rtol=RTOL,
                               build_sweeps=BUILD_SWEEPS, apply_sweeps_lower=APPLY_SWEEPS,
                               apply_sweeps_upper=APPLY_SWEEPS, mode=args.mode,
                               raise_on_noconv=True, zero_guess=True)

    # ---- per-kernel rooflines (the dominant kernel by solve time share),
    # isolated, before the timed region: a few hundred ms of GPU work that
    # also brings the clocks up from the idle of the host-only setup (with
    # only the warm-up solves before it, the 34 ms timed region of a 20-solve
    # run sampled 2,002 MHz against the 2,070 maximum)
    fk = ab.Factors(pat, "f32")
    fk.build(A, BUILD_SWEEPS, args.mode)
    kern = kernel_rooflines(torch, ab, pat, A, fk, s, peak, args.mode)
    del fk

    # the build inside every BUILD_TIMED_EVERY-th timed solve records CUDA
    # events around its sweep kernels on the solve's stream: the dominant
    # kernel's duration is read from the timed region itself.  Not every
    # solve: the two events sit between kernels chained by programmatic
    # dependent launch and cost a solve that records them about 10 us
    # (1,673 against 1,663 us per solve with and without them)
    fac.timing(True)
    for _ in range(args.warmup):
        res = solve()
    fac.timing(False)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    evs = _events(torch, 2)
    barrier()
    clocks.start()
    clocks.begin()
    l0 = ab.kernel_launches()
    evs[0].record(stream)
    iters, sweep_ms = [], []
    for k in range(args.steps):
        timed = k % BUILD_TIMED_EVERY == 0
        if timed:
            fac.timing(True)
        res = solve()
        if timed:
            sweep_ms.append(fac.sweep_ms())
            fac.timing(False)
        iters.append(res.iters)
    evs[1].record(stream)
    barrier()
    clocks.end()
    launches = ab.kernel_launches() - l0
    clk = clocks.stop()
    total_ms = max_over_ranks(torch, evs[0].elapsed_time(evs[1]), dev)
    value = job_rate(args.steps, world, total_ms)

    # ---- end to end: A and b from pinned host memory, x back, every step.
    # Double-buffered like a serving loop: the next step's A and b stream in
    # and the previous step's x streams out on a copy stream while the current
    # step solves (every step's inputs and result still cross the host link
    # inside the timed region; the last x is waited for before it closes).
    hA = torch.from_numpy(s.vals).pin_memory()
    hb = torch.from_numpy(s.b).pin_memory()
    hx = [torch.empty_like(hb).pin_memory(), torch.empty_like(hb).pin_memory()]
    dA = [torch.empty_like(A), torch.empty_like(A)]
    db = [torch.empty_like(b), torch.empty_like(b)]
    dx = [torch.empty_like(b), torch.empty_like(b)]
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    solved = [torch.cuda.Event(), torch.cuda.Event()]

    def h2d(k):
        with torch.cuda.stream(copy_stream):
            dA[k % 2].copy_(hA, non_blocking=True)
            db[k % 2].copy_(hb, non_blocking=True)
            ready[k % 2].record(copy_stream)

    def e2e_steps(nsteps):
        # copy-stream order: h2d(k+1), d2h(k), h2d(k+2), ...: step k+2, which
        # overwrites dx[k % 2], waits for h2d(k+2) and so for d2h(k)
        h2d(0)
        for k in range(nsteps):
            if k + 1 < nsteps:
                h2d(k + 1)      # buffer (k+1) % 2 was last read by step k-1, finished
            stream.wait_event(ready[k % 2])
            ab.fgmres_solve(pat, dA[k % 2], fac, db[k % 2], dx[k % 2], restart=RESTART,
                            rtol=RTOL, build_sweeps=BUILD_SWEEPS,
                            apply_sweeps_lower=APPLY_SWEEPS, apply_sweeps_upper=APPLY_SWEEPS,
                            mode=args.mode, raise_on_noconv=True, zero_guess=True)
            solved[k % 2].record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(solved[k % 2])
                hx[k % 2].copy_(dx[k % 2], non_blocking=True)
        stream.wait_stream(copy_stream)

    e2e_steps(2)
    torch.cuda.synchronize()
    e0, e1 = _events(torch, 2)
    barrier()
    e0.record(stream)
    e2e_steps(args.steps)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(torch, e0.elapsed_time(e1), dev)
    e2e = {"value": job_rate(args.steps, world, e2e_ms), "unit": "solves/s",
           "h2d_bytes_per_step": hA.numel() * 8 + hb.numel() * 8,
           "d2h_bytes_per_step": hx[0].numel() * 8}

    it = statistics.median(iters)
    # launches of each kernel per solve (it Arnoldi steps, 2 residuals); every
    # Arnoldi step forms w = A z_j inside the kernel that also takes the
    # Gram-Schmidt dots, so the stand-alone product (timed above for its
    # roofline) runs in no step of the solve
    spmv_steps = 0
    if args.mode == "async":
        per_solve = {"spmv_f64": spmv_steps, "build_sweeps_f32": 1, "build_prepare_f32": 1,
                     "lower_sweeps_f32": it, "upper_sweeps_f32": it}
    else:
        per_solve = {"spmv_f64": spmv_steps, "build_sweep_f32": BUILD_SWEEPS, "build_prepare_f32": 1,
                     "lower_sweep_f32": it * (APPLY_SWEEPS - 1),
                     "upper_sweep_f32": it * (APPLY_SWEEPS - 1)}
    share = {k: kern[k]["us"] * per_solve[k] for k in kern}
    dom = max(share, key=share.get)
    dk = kern[dom]
    # the build sweeps' duration from the timed solves themselves (events
    # around the sweep kernels of each solve's build); other kernels: isolated
    timing = "isolated"
    dom_us = dk["us"]
    if dom.startswith("build_sweep"):
        per_build = 1 if args.mode == "async" else BUILD_SWEEPS   # launches per build
        dom_us = statistics.mean(sweep_ms) * 1e3 / per_build
        timing = "timed region"
    dom_gbs = dk["bytes"] / (dom_us * 1e-6) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(dom_gbs, 1), "peak": peak,
            "unit": "GB/s", "frac": round(dom_gbs / peak, 4),
            "traffic": PROFILED_TRAFFIC.get(dom), "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": dk["bytes"], "sweeps_per_launch": dk["sweeps"],
            "us_per_launch": round(dom_us, 2), "timing": timing,
            "timed_launches": len(sweep_ms) if timing == "timed region" else None,
            "us_per_launch_isolated": round(dk["us"], 2)}
    kernels = {k: {"us_per_call": round(v["us"], 2), "GBs": round(v["GBs"], 1),
                   "frac_of_measured_peak": round(v["frac"], 4),
                   "us_per_solve": round(share[k], 1)} for k, v in kern.items()}

    # ---- variants (same workload, fewer steps)
    variants = {}
    if args.variants:
        for dt, md in (("f64", "sync"), ("f32", "sync"), ("f32", "async"), ("bf16", "sync"),
                       ("f64", "async")):
            fv = ab.Factors(pat, dt)
            xv = torch.zeros_like(b)

            def sv():
                return ab.fgmres_solve(pat, A, fv, b, xv, restart=RESTART, rtol=RTOL,
                                       build_sweeps=BUILD_SWEEPS,
                                       apply_sweeps_lower=APPLY_SWEEPS,
                                       apply_sweeps_upper=APPLY_SWEEPS, mode=md, zero_guess=True)
            r = sv()
            sv()
            torch.cuda.synchronize()
            a0, a1 = _events(torch, 2)
            a0.record(stream)
            for _ in range(5):
                r = sv()
            a1.record(stream)
            torch.cuda.synchronize()
            variants[f"{dt}_{md}"] = {"solves_per_s": round(5 / (a0.elapsed_time(a1) * 1e-3), 1),
                                      "iters": r.iters, "rel_resid_true": r.rel_resid_true,
                                      "x": xv.cpu().numpy()}

    # ---- latency: >= 200 solves, each between its own events (outside the
    # timed region, so that p99 is a percentile and not the maximum)
    nlat = max(200, args.steps)
    lev = _events(torch, nlat + 1)
    torch.cuda.synchronize()
    lev[0].record(stream)
    for k in range(nlat):
        solve()
        lev[k + 1].record(stream)
    torch.cuda.synchronize()
    lat_ms = sorted(lev[k].elapsed_time(lev[k + 1]) for k in range(nlat))

    # ---- the other workloads of the benchmark: viscous-like grid in both
    # orderings, the uneven batch, the serving stream
    extras = {}
    if rank == 0 and world == 1 and args.extras:
        extras["viscous"] = viscous_rcm_vs_line()
        extras["batched"] = run_batched(args)
        # five timed runs per configuration: a 20-request run lasts about 0.1 s,
        # and single runs lost up to 40% to stalls of the shared host
        extras["serving"] = run_serving(args, n_requests=20, rates=(0.5, 1.0), reps=5)

    cpu = None
    x_gpu = x.cpu().numpy()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np
        vis = None
        if args.extras:
            import abilu_inputs as gen
            vis = gen.workload("viscous_1024x256_rcm")
        cpu, x_or, r_or = cpu_baseline(s, viscous=vis)
        nrm = float(np.linalg.norm(x_or))
        err = {"rel_l2": float(np.linalg.norm(x_gpu - x_or)) / nrm,
               "rel_max": float(np.abs(x_gpu - x_or).max() / np.abs(x_or).max()),
               "oracle_iters": r_or.iters, "oracle_rel_resid_true": r_or.rel_resid_true}
        for name, v in variants.items():
            v["err_vs_oracle"] = _r(float(np.linalg.norm(v.pop("x") - x_or)) / nrm)
    for v in variants.values():
        v.pop("x", None)

    if rank == 0:
        p50 = statistics.median(lat_ms)
        p99 = lat_ms[min(len(lat_ms) - 1, int(round(0.99 * (len(lat_ms) - 1))))]
        line = {"metric": METRIC, "value": round(value, 2), "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "cells": s.n, "blocks": s.nnzb,
                           "factor_dtype": args.dtype, "mode": args.mode,
                           "build_sweeps": BUILD_SWEEPS, "apply_sweeps": APPLY_SWEEPS,
                           "restart": RESTART, "rtol": RTOL, "iters": iters[-1],
                           "rel_resid_true": res.rel_resid_true,
                           "parallelism": f"replicas{world}",
                           "l2": "inputs larger than L2 (A = %.0f MB)" % (s.nnzb * 128 / 1e6)},
                "latency_ms": {"p50": round(p50, 4), "p99": round(p99, 4), "samples": nlat},
                "err_vs_oracle": ({k: _r(v) for k, v in err.items()} if cpu else None),
                "gpu_launches": int(launches),
                "e2e": {k: (round(v, 2) if isinstance(v, float) else v) for k, v in e2e.items()},
                "roofline": roof, "kernels": kernels, "variants": variants,
                "clocks": clk, "cpu_baseline": cpu, **extras}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f64"])
    ap.add_argument("--mode", default="async", choices=["sync", "async"])
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the viscous, batched and serving sections of the default line")
    ap.add_argument("--kernels-only", action="store_true")
    ap.add_argument("--profile-solves", type=int, default=0)
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="warm-up plus this many solves of the 64-system batch, for ncu")
    ap.add_argument("--profile-mg", type=int, default=0,
                    help="warm-up plus this many multigrid-preconditioned solves, for ncu")
    ap.add_argument("--batched", action="store_true", help="only the batched workload")
    ap.add_argument("--serving", action="store_true", help="only the serving workload")
    ap.add_argument("--viscous", action="store_true", help="only the viscous-like workload")
    ap.add_argument("--scalar", action="store_true",
                    help="only the block vs scalar (Chow-Patel) ILU(0) comparison")
    ap.add_argument("--continuation", action="store_true",
                    help="only the pseudo-time continuation of a steady model problem")
    ap.add_argument("--multigrid", action="store_true",
                    help="only block ILU as a multigrid smoother (V-cycle preconditioner)")
    ap.add_argument("--parilut", action="store_true",
                    help="only the threshold block ILU against block ILU(0)")
    ap.add_argument("--batch-build-sweeps", type=int, default=4)
    ap.add_argument("--batch-apply-sweeps", type=int, default=3)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernels_only:
        return run_kernels_only(args)
    if args.profile_solves:
        return run_profile_solves(args)
    if args.profile_mg:
        return run_profile_mg(args)
    if args.profile_batch:
        return run_profile_batch(args)
    if args.batched:
        print(json.dumps(run_batched(args)))
        return 0
    if args.serving:
        print(json.dumps(run_serving(args)))
        return 0
    if args.viscous:
        print(json.dumps(run_viscous(args)))
        return 0
    if args.continuation:
        print(json.dumps(run_continuation(args)))
        return 0
    if args.scalar:
        print(json.dumps(run_scalar_vs_block(args)))
        return 0
    if args.multigrid:
        print(json.dumps(run_multigrid(args)))
        return 0
    if args.parilut:
        print(json.dumps(run_parilut(args)))
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
