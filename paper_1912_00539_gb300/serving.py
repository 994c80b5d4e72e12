"""Continuous solve server for sequences of value updates on fixed patterns.

A request is one block pattern and a sequence of value updates (A_k, b_k): the
successive pseudo-time steps of one flow computation (Sec. 2: the Jacobian's
pattern is fixed, its values change every step, the CFL number ramps up).
The server

* admits a request when its device footprint fits in the HBM budget and a
  slot is free (first come, first served);
* keeps the request's pattern, factors and Krylov workspace on the device for
  its whole life; update k+1 warm-starts from the factors of update k
  (init = previous, Sec. 3.3: the factors of the previous time step are a
  natural initial guess);
* runs the admitted requests at the same time, each on its own CUDA stream
  from its own host thread, so their kernels overlap on the GPU; a request
  that arrives while others run is admitted as soon as a slot and memory free
  up, not when the others finish;
* releases the slot when the request's last update is solved.

Device memory of finished requests is released in bulk when the server goes
idle (cudaFree synchronises the whole device and would stall the others).
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import abilu as ab


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the stream
    rowptr: np.ndarray
    colind: np.ndarray
    updates: list                  # [(vals (nnzb,4,4) float64, b (n,4) float64), ...]

    @property
    def n(self):
        return len(self.rowptr) - 1

    @property
    def nnzb(self):
        return len(self.colind)


@dataclass
class RequestResult:
    rid: int
    n: int
    arrival: float
    admitted: float
    finished: float
    update_ms: list = field(default_factory=list)   # solve time of each update
    iters: list = field(default_factory=list)
    rel_resid: list = field(default_factory=list)
    x: list = field(default_factory=list)           # host solutions (if kept)

    @property
    def latency(self):
        return self.finished - self.arrival


def footprint_bytes(n: int, nnzb: int, dtype: str = "f32", restart: int = 30) -> int:
    """Device bytes one request holds: A, b, x, pattern arrays (including the
    build's work list and records), factors (two iterates, inverses, U_ii, and
    for FP32/BF16 the FP32 copy of A, for FP32 the Dinv-scaled upper blocks), sweep
    vectors and the Krylov basis (V: restart+1 vectors, Z: restart, w)."""
    f = {"f64": 8, "f32": 4, "bf16": 2}[dtype]
    vec = 32 * n
    a = 128 * nnzb
    pattern = 4 * (2 * nnzb + 7 * n) + 8 * nnzb + 16 * nnzb + 8 * nnzb + 4 * nnzb + 32 * nnzb
    narrow = (64 * nnzb + 16 * n if f < 8 else 0) + (8 * f * nnzb if f == 4 else 0)
    factors = 2 * 16 * f * nnzb + 3 * 16 * f * n + narrow + 4 * vec
    krylov = (2 * restart + 2) * vec
    return a + 2 * vec + pattern + factors + krylov


class Server:
    def __init__(self, hbm_budget_bytes: float, slots: int = 8, dtype: str = "f32",
                 mode: str = "async", build_sweeps: int = 4, apply_sweeps: int = 3,
                 restart: int = 30, rtol: float = 1e-6, keep_solutions: bool = False):
        self.budget = float(hbm_budget_bytes)
        self.slots = int(slots)
        self.dtype = dtype
        self.mode = mode
        self.build_sweeps = build_sweeps
        self.apply_sweeps = apply_sweeps
        self.restart = restart
        self.rtol = rtol
        self.keep = keep_solutions

    def run(self, requests):
        """Serve `requests` (arrival times relative to now); returns results in
        request order and the wall time of the whole stream."""
        import torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        # the producer hands over each update in pinned host memory
        host = {r.rid: [(torch.from_numpy(np.ascontiguousarray(v)).pin_memory(),
                         torch.from_numpy(np.ascontiguousarray(b)).pin_memory())
                        for v, b in r.updates] for r in reqs}
        lock = threading.Condition()
        state = {"used": 0.0, "active": 0, "next": 0, "arrived": 0}
        results = {}
        graveyard = []
        errors = []
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def serve(r: Request, admitted: float):
            stream = torch.cuda.Stream()
            res = RequestResult(r.rid, r.n, r.arrival, admitted, 0.0)
            with torch.cuda.stream(stream):
                rowptr = torch.from_numpy(r.rowptr).cuda(non_blocking=False)
                colind = torch.from_numpy(r.colind).cuda(non_blocking=False)
                pat = ab.Pattern(rowptr, colind, stream=stream)
                fac = ab.Factors(pat, self.dtype)
                A = torch.empty((r.nnzb, 4, 4), dtype=torch.float64, device="cuda")
                b = torch.empty((r.n, 4), dtype=torch.float64, device="cuda")
                x = torch.zeros_like(b)
                xh = torch.empty_like(b, device="cpu").pin_memory()
                for k, (hA, hb) in enumerate(host[r.rid]):
                    ts = time.perf_counter()
                    A.copy_(hA, non_blocking=True)
                    b.copy_(hb, non_blocking=True)
                    x.zero_()
                    sr = ab.fgmres_solve(pat, A, fac, b, x, restart=self.restart, rtol=self.rtol,
                                         build_sweeps=self.build_sweeps,
                                         apply_sweeps_lower=self.apply_sweeps,
                                         apply_sweeps_upper=self.apply_sweeps, mode=self.mode,
                                         init="a" if k == 0 else "previous", stream=stream)
                    xh.copy_(x, non_blocking=True)
                    stream.synchronize()
                    res.update_ms.append(1e3 * (time.perf_counter() - ts))
                    res.iters.append(sr.iters)
                    res.rel_resid.append(sr.rel_resid_true)
                    if self.keep:
                        res.x.append(xh.numpy().copy())
            res.finished = now()
            return res, (pat, fac, A, b, x, rowptr, colind)

        def worker():
            while True:
                with lock:
                    while True:
                        i = state["next"]
                        if i >= len(reqs):
                            return
                        r = reqs[i]
                        fp = footprint_bytes(r.n, r.nnzb, self.dtype, self.restart)
                        arrived = now() >= r.arrival
                        fits = state["used"] + fp <= self.budget or state["active"] == 0
                        if arrived and fits and state["active"] < self.slots:
                            state["next"] += 1
                            state["used"] += fp
                            state["active"] += 1
                            break
                        wait = max(0.0, r.arrival - now()) if not arrived else None
                        lock.wait(timeout=wait if wait else 0.05)
                admitted = now()
                try:
                    res, objs = serve(r, admitted)
                except Exception as e:  # surfaced after the run
                    errors.append(e)
                    res, objs = None, ()
                with lock:
                    if res is not None:
                        results[r.rid] = res
                    graveyard.append(objs)
                    state["used"] -= fp
                    state["active"] -= 1
                    lock.notify_all()

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.slots)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        wall = now()
        torch.cuda.synchronize()
        graveyard.clear()
        if errors:
            raise errors[0]
        return [results[r.rid] for r in requests], wall


def summarize(results, wall):
    lat = np.array([r.latency for r in results]) * 1e3
    upd = np.concatenate([np.array(r.update_ms) for r in results])
    n_upd = sum(len(r.update_ms) for r in results)
    return {"requests": len(results), "updates": n_upd,
            "solves_per_s": n_upd / wall if wall > 0 else 0.0,
            "request_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                   "p99": float(np.percentile(lat, 99))},
            "solve_latency_ms": {"p50": float(np.percentile(upd, 50)),
                                 "p99": float(np.percentile(upd, 99))},
            "max_iters": int(max(max(r.iters) for r in results)),
            "max_rel_resid": float(max(max(r.rel_resid) for r in results)),
            "wall_s": wall}
