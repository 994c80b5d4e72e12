"""Empirical autotuner for the preconditioner's sweep counts and mode.

How many build sweeps and triangular sweeps pay off depends on the matrices
(the paper's Tables 1-3 show iteration counts moving with both, and a setting
that is best for one flow case is poor for another), and the best
synchronous/asynchronous choice depends on the GPU's scheduling.  The tuner
times complete solves (CUDA events) over a grid of candidates, keeps the
fastest one that converges, and caches the choice in a JSON file keyed by GPU
name, factor dtype and size bucket (log2 of the number of cells), so later
runs of similar workloads reuse it.

The kernels' launch shapes are fixed by the design: 4 threads per block row
(one per row of a 4x4 block: 16-byte FP32 rows, quad shuffles for the block
products) and 64 rows per CTA (the chunk unit of batches); the candidates
vary what the matrices make variable.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import asdict, dataclass

DEFAULT_GRID = [(b, a, m) for b in (2, 4, 6) for a in (2, 3, 4) for m in ("sync", "async")]


@dataclass
class Choice:
    build_sweeps: int
    apply_sweeps: int
    mode: str
    ms: float
    iters: int


def _key(gpu: str, dtype: str, cells: int) -> str:
    return f"{gpu}|{dtype}|2^{int(round(math.log2(max(cells, 1))))}"


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
         cache_path: str | None = None, refresh: bool = False) -> Choice:
    """solve(build_sweeps, apply_sweeps, mode) -> list of SolveResult (or one).
    Returns the fastest converging candidate; reads/writes `cache_path`."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(gpu, dtype, cells)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache and not refresh:
        return Choice(**cache[key])
    best = None
    for b, a, m in grid or DEFAULT_GRID:
        ms, res = _timed(torch, lambda: solve(b, a, m), repeats)
        res = res if isinstance(res, list) else [res]
        if not all(r.converged for r in res):
            continue
        c = Choice(b, a, m, ms, max(r.iters for r in res))
        if best is None or c.ms < best.ms:
            best = c
    if best is None:
        raise RuntimeError("autotune: no candidate converged")
    if cache_path:
        cache[key] = asdict(best)
        tmp = f"{cache_path}.tmp{os.getpid()}.{time.time_ns()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return best


def tune_batch(batch, cells: int, restart: int = 30, rtol: float = 1e-6, **kw) -> Choice:
    return tune(lambda b, a, m: batch.solve(restart=restart, rtol=rtol, build_sweeps=b,
                                            apply_sweeps_lower=a, apply_sweeps_upper=a, mode=m),
                cells, batch.dtype, **kw)
