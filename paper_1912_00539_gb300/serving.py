"""Continuous-batching solve server for sequences of value updates on fixed
patterns.

A request is one block pattern and a sequence of value updates (A_k, b_k): the
successive pseudo-time steps of one flow computation (Sec. 2: the Jacobian's
pattern is fixed, its values change every step, the CFL number ramps up).

The server is a scheduler over the library's native continuous-batching
engine (abilu_server_*, a preallocated device arena sized to the HBM budget):

* a request is admitted when it has arrived and the arena has room for it
  (first come, first served); its pattern is analysed once, on admission;
* every step solves one update of every admitted request in shared launches
  (one batched build and FGMRES solve); update k+1 of a request is ready when
  update k is solved, and its build warm-starts from update k's factors
  (Sec. 6 setup: the factors of the previous pseudo-time step are a natural
  initial guess);
* a request that arrives while a step runs joins at the next step, when the
  arena has room, without waiting for the others to finish;
* a finished request leaves at once: its pattern analysis is released and its
  share of the arena serves the next admission (no memory is held back).

`serve_one_at_a_time` is the baseline: the same requests solved in arrival
order, one request and one update at a time, through the single-system API.
"""
from __future__ import annotations

import collections
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
    update_ms: list = field(default_factory=list)   # ready -> solved, each update
    iters: list = field(default_factory=list)
    rel_resid: list = field(default_factory=list)
    x: list = field(default_factory=list)           # host solutions (if kept)
    steps: list = field(default_factory=list)       # systems in the step of each update

    @property
    def latency(self):
        return self.finished - self.arrival


def _pinned(a):
    """A pinned host tensor of a (numpy arrays are copied; tensors are taken
    as they are)."""
    import torch
    if isinstance(a, torch.Tensor):
        return a
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def pattern_bytes(n: int, nnzb: int) -> int:
    """Device bytes of one admitted request's own pattern analysis (row and
    block index arrays, product pairs, 32-byte work records), outside the
    arena; pairs and work items are bounded by the blocks."""
    return 4 * (9 * n + 6 * nnzb) + 8 * nnzb + 48 * nnzb + 4096


def arena_cells_for_budget(budget_bytes: float, dtype: str = "f32", restart: int = 30,
                           blocks_per_cell: float = 4.2, max_systems: int = 64) -> int:
    """The largest arena (rows, a multiple of 64, with blocks_per_cell blocks
    per row) whose device bytes fit budget_bytes (0 if none does)."""
    def fits(cells):
        try:
            return ab.server_arena_bytes(cells, int(blocks_per_cell * cells), max_systems, dtype,
                                         restart) <= budget_bytes
        except ab.AbiluError:     # beyond the engine's index range
            return False
    if not fits(64):
        return 0
    lo, hi = 64, 128
    while fits(hi):
        lo, hi = hi, hi * 2
    while hi - lo > 64:
        mid = (lo + hi) // 2 // 64 * 64
        if mid <= lo:
            break
        if fits(mid):
            lo = mid
        else:
            hi = mid
    return lo


class Server:
    """Continuous batching of requests in one arena (see the module notes).

    hbm_budget_bytes: device memory the server may hold: the arena gets
    (1 - pattern_reserve) of it, the rest bounds the admitted requests' own
    pattern analyses."""

    def __init__(self, hbm_budget_bytes: float, dtype: str = "f32", mode: str = "async",
                 build_sweeps: int = 4, apply_sweeps: int = 3, restart: int = 30,
                 rtol: float = 1e-6, max_systems: int = 64, keep_solutions: bool = False,
                 blocks_per_cell: float = 4.2, pattern_reserve: float = 0.1):
        self.budget = float(hbm_budget_bytes)
        self.dtype = dtype
        self.mode = mode
        self.build_sweeps = build_sweeps
        self.apply_sweeps = apply_sweeps
        self.restart = restart
        self.rtol = rtol
        self.max_systems = max_systems
        self.keep = keep_solutions
        self.pattern_budget = pattern_reserve * self.budget
        self.cells = arena_cells_for_budget((1.0 - pattern_reserve) * self.budget, dtype, restart,
                                            blocks_per_cell, max_systems)
        self.blocks = int(blocks_per_cell * self.cells)
        self.arena_bytes = ab.server_arena_bytes(self.cells, self.blocks, max_systems, dtype,
                                                 restart)
        self.engine = None
        self.memory_samples = []    # (time, device bytes in use) before every step

    def _engine(self):
        if self.engine is None:
            self.engine = ab.NativeServer(self.cells, self.blocks, self.max_systems, self.dtype,
                                          self.restart)
        return self.engine

    def run(self, requests):
        """Serve `requests` (arrival times relative to now); returns results in
        request order and the wall time of the whole stream."""
        import torch
        eng = self._engine()
        reqs = sorted(requests, key=lambda r: r.arrival)
        # the producer hands over each update in pinned host memory
        host = {r.rid: [(_pinned(v), _pinned(b)) for v, b in r.updates] for r in reqs}
        xout = {r.rid: torch.empty((r.n, 4), dtype=torch.float64).pin_memory() for r in reqs}
        queue = collections.deque(reqs)
        active = []
        results = {}
        pat_used = 0.0
        opts = dict(restart=self.restart, rtol=self.rtol, build_sweeps=self.build_sweeps,
                    apply_sweeps_lower=self.apply_sweeps, apply_sweeps_upper=self.apply_sweeps,
                    mode=self.mode)
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        while queue or active:
            t = now()
            while queue and queue[0].arrival <= t:
                r = queue[0]
                pb = pattern_bytes(r.n, r.nnzb)
                if active and pat_used + pb > self.pattern_budget:
                    break
                sid = eng.add(torch.from_numpy(r.rowptr).cuda(), torch.from_numpy(r.colind).cuda())
                if sid is None:
                    if not active:
                        raise ValueError(f"request {r.rid} ({r.n} cells) does not fit the arena "
                                         f"({self.cells} cells)")
                    break          # first come, first served: wait for a departure
                queue.popleft()
                pat_used += pb
                active.append({"r": r, "id": sid, "k": 0, "ready": r.arrival, "pb": pb,
                               "res": RequestResult(r.rid, r.n, r.arrival, now(), 0.0)})
            if not active:
                wait = queue[0].arrival - now()
                if wait > 0:
                    time.sleep(min(wait, 0.001))
                continue
            free, total = torch.cuda.mem_get_info()
            self.memory_samples.append((now(), total - free))
            out = eng.step([a["id"] for a in active],
                           [host[a["r"].rid][a["k"]][0] for a in active],
                           [host[a["r"].rid][a["k"]][1] for a in active],
                           [xout[a["r"].rid] for a in active], **opts)
            tend = now()
            k = len(active)
            for a, o in zip(active, out):
                res = a["res"]
                res.update_ms.append(1e3 * (tend - a["ready"]))
                res.iters.append(o.iters)
                res.rel_resid.append(o.rel_resid_true)
                res.steps.append(k)
                if self.keep:
                    res.x.append(xout[a["r"].rid].numpy().copy())
                a["k"] += 1
                a["ready"] = tend
            still = []
            for a in active:
                if a["k"] == len(a["r"].updates):
                    eng.remove(a["id"])
                    pat_used -= a["pb"]
                    a["res"].finished = tend
                    results[a["r"].rid] = a["res"]
                else:
                    still.append(a)
            active = still
        wall = now()
        return [results[r.rid] for r in requests], wall

    def close(self):
        self.engine = None


def serve_one_at_a_time(requests, dtype: str = "f64", mode: str = "sync", build_sweeps: int = 4,
                        apply_sweeps: int = 3, restart: int = 30, rtol: float = 1e-6,
                        keep_solutions: bool = False):
    """The baseline: requests in arrival order, one at a time, each update
    solved by fgmres_solve on the request's own handles (warm-started from the
    previous update's factors), inputs from pinned host memory."""
    import torch
    reqs = sorted(requests, key=lambda r: r.arrival)
    host = {r.rid: [(_pinned(v), _pinned(b)) for v, b in r.updates] for r in reqs}
    results = {}
    t0 = time.perf_counter()

    def now():
        return time.perf_counter() - t0

    for r in reqs:
        while now() < r.arrival:
            time.sleep(min(r.arrival - now(), 0.001))
        res = RequestResult(r.rid, r.n, r.arrival, now(), 0.0)
        rowptr = torch.from_numpy(r.rowptr).cuda()
        colind = torch.from_numpy(r.colind).cuda()
        pat = ab.Pattern(rowptr, colind)
        fac = ab.Factors(pat, dtype)
        A = torch.empty((r.nnzb, 4, 4), dtype=torch.float64, device="cuda")
        b = torch.empty((r.n, 4), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        xh = torch.empty((r.n, 4), dtype=torch.float64).pin_memory()
        ready = r.arrival
        for k, (v, bh) in enumerate(host[r.rid]):
            A.copy_(v, non_blocking=True)
            b.copy_(bh, non_blocking=True)
            sr = ab.fgmres_solve(pat, A, fac, b, x, restart=restart, rtol=rtol,
                                 build_sweeps=build_sweeps, apply_sweeps_lower=apply_sweeps,
                                 apply_sweeps_upper=apply_sweeps, mode=mode,
                                 init="a" if k == 0 else "previous", zero_guess=True)
            xh.copy_(x)
            t = now()
            res.update_ms.append(1e3 * (t - ready))
            ready = t
            res.iters.append(sr.iters)
            res.rel_resid.append(sr.rel_resid_true)
            res.steps.append(1)
            if keep_solutions:
                res.x.append(xh.numpy().copy())
        res.finished = now()
        results[r.rid] = res
        del fac, pat
    return [results[r.rid] for r in requests], now()


def summarize(results, wall):
    lat = np.array([r.latency for r in results]) * 1e3
    upd = np.concatenate([np.array(r.update_ms) for r in results])
    n_upd = sum(len(r.update_ms) for r in results)
    steps = np.concatenate([np.array(r.steps) for r in results]) if results[0].steps else None
    out = {"requests": len(results), "updates": n_upd,
           "solves_per_s": n_upd / wall if wall > 0 else 0.0,
           "request_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                  "p99": float(np.percentile(lat, 99))},
           "solve_latency_ms": {"p50": float(np.percentile(upd, 50)),
                                "p99": float(np.percentile(upd, 99)), "samples": int(len(upd))},
           "max_iters": int(max(max(r.iters) for r in results)),
           "max_rel_resid": float(max(max(r.rel_resid) for r in results)),
           "wall_s": wall}
    if steps is not None:
        out["systems_per_step"] = {"mean": float(steps.mean()), "max": int(steps.max())}
    return out
