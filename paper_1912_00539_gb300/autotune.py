"""Empirical autotuner for the preconditioner's sweep counts, mode and the
asynchronous build's launch shape.

How many build sweeps and triangular sweeps pay off depends on the matrices
(the paper's Tables 1-3 show iteration counts moving with both, and a setting
that is best for one flow case is poor for another), and the best
synchronous/asynchronous choice depends on the GPU's scheduling.  The tuner
times complete solves (CUDA events) over a grid of candidates, keeps the
fastest one that converges, and caches the choice in a JSON file keyed by GPU
name, factor dtype, size bucket (log2 of the number of cells) and, when the
caller gives it, the CFL range of the systems (the pseudo-time step sets the
diagonal dominance that decides how many sweeps a build needs), so later runs
of similar workloads reuse it.

Launch shape: the asynchronous block build hands out its work in tickets of
`build_chunk` work blocks per warp (abilu_factors_set_build_chunk); small
tickets balance the load, and leave a lower ILU residual after the same
sweeps (the tickets in flight span fewer blocks, so more of the rows a block
reads are already updated in the current sweep), but contend on the one
ticket counter; the best size moves with the system's size and with the
sweep count, so it is a candidate of the asynchronous mode.  The other kernels' shapes are fixed by
the data: 4 threads per block row (one per row of a 4x4 block: a 16-byte FP32
or 32-byte FP64 row per thread, quad shuffles for the block products; 8 or 16
threads would split a row below one element per thread) and 64 rows per CTA
(the chunk unit of batches, the skip flags and the per-system reductions).
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import asdict, dataclass

BUILD_CHUNKS = (64, 128, 256)
DEFAULT_GRID = ([(b, a, "sync", 0) for b in (2, 4, 6) for a in (2, 3, 4)] +
                [(b, a, "async", c) for b in (2, 4, 6) for a in (2, 3, 4) for c in BUILD_CHUNKS])


@dataclass
class Choice:
    build_sweeps: int
    apply_sweeps: int
    mode: str
    ms: float
    iters: int
    build_chunk: int = 0     # work blocks per ticket of the async build (0: the default)


def cfl_bucket(cfl_lo: float, cfl_hi: float) -> str:
    """The decades a set of systems' CFL numbers span, e.g. 'cfl1e1-1e4'."""
    lo = int(math.floor(math.log10(max(cfl_lo, 1e-300))))
    hi = int(math.ceil(math.log10(max(cfl_hi, 1e-300))))
    return f"cfl1e{lo}-1e{hi}"


def _key(gpu: str, dtype: str, cells: int, cond: str | None = None) -> str:
    k = f"{gpu}|{dtype}|2^{int(round(math.log2(max(cells, 1))))}"
    return f"{k}|{cond}" if cond else k


def _timed(torch, fn, repeats):
    fn()  # warm-up (and convergence check)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(repeats):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / repeats, out


def tune(solve, cells: int, dtype: str = "f32", grid=None, repeats: int = 2,
         cache_path: str | None = None, refresh: bool = False,
         cond: str | None = None) -> Choice:
    """solve(build_sweeps, apply_sweeps, mode, build_chunk) -> list of
    SolveResult (or one).  Returns the fastest converging candidate;
    reads/writes `cache_path`; `cond` (e.g. cfl_bucket(...)) refines the key."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(gpu, dtype, cells, cond)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache and not refresh:
        return Choice(**cache[key])
    best = None
    for b, a, m, c in grid or DEFAULT_GRID:
        ms, res = _timed(torch, lambda: solve(b, a, m, c), repeats)
        res = res if isinstance(res, list) else [res]
        if not all(r.converged for r in res):
            continue
        ch = Choice(b, a, m, ms, max(r.iters for r in res), c)
        if best is None or ch.ms < best.ms:
            best = ch
    if best is None:
        raise RuntimeError("autotune: no candidate converged")
    if cache_path:
        cache[key] = asdict(best)
        tmp = f"{cache_path}.tmp{os.getpid()}.{time.time_ns()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return best


def tune_batch(batch, cells: int, restart: int = 30, rtol: float = 1e-6,
               cfl_range: tuple | None = None, **kw) -> Choice:
    """Tune a batch (ab.Batch); the chosen build chunk stays set on it."""
    def solve(b, a, m, c):
        batch.set_build_chunk(c)
        return batch.solve(restart=restart, rtol=rtol, build_sweeps=b, apply_sweeps_lower=a,
                           apply_sweeps_upper=a, mode=m)
    cond = cfl_bucket(*cfl_range) if cfl_range else None
    choice = tune(solve, cells, batch.dtype, cond=cond, **kw)
    batch.set_build_chunk(choice.build_chunk)
    return choice


def tune_system(pattern, A, factors, b, x, restart: int = 30, rtol: float = 1e-6,
                cfl: float | None = None, **kw) -> Choice:
    """Tune one system's solve (fgmres_solve on the given handles); the
    chosen build chunk stays set on `factors`."""
    from . import abilu as ab

    def solve(nb, na, m, c):
        factors.set_build_chunk(c)
        return ab.fgmres_solve(pattern, A, factors, b, x, restart=restart, rtol=rtol,
                               build_sweeps=nb, apply_sweeps_lower=na, apply_sweeps_upper=na,
                               mode=m, zero_guess=True)
    cond = cfl_bucket(cfl, cfl) if cfl else None
    choice = tune(solve, pattern.n, factors.dtype, cond=cond, **kw)
    factors.set_build_chunk(choice.build_chunk)
    return choice
