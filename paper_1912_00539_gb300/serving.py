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
                 blocks_per_cell: float = 4.2, pattern_reserve: float = 0.1, groups: int = 4):
        self.groups = int(groups)
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
        # each group's arena: an equal share of the rest of the budget
        self.cells = arena_cells_for_budget((1.0 - pattern_reserve) * self.budget / self.groups,
                                            dtype, restart, blocks_per_cell, max_systems)
        self.blocks = int(blocks_per_cell * self.cells)
        self.arena_bytes = self.groups * ab.server_arena_bytes(self.cells, self.blocks,
                                                               max_systems, dtype, restart)
        self.engines = None
        self.memory_samples = []    # (time, device bytes in use) before every step

    def _engine(self):
        if self.engines is None:
            self.engines = [ab.NativeServer(self.cells, self.blocks, self.max_systems, self.dtype,
                                            self.restart) for _ in range(self.groups)]
        return self.engines

    def run(self, requests, lookahead: int = 16):
        """Serve `requests` (arrival times relative to now); returns results in
        request order and the wall time of the whole stream.

        Every group is an arena of its own, stepped by its own host thread on
        its own stream, so that one group's host-to-device copies of a step's
        values overlap another group's solve (the copies of a step must
        follow the previous step: update k+1 exists once update k is solved).
        Admission is first come, first served: the head of the queue joins the
        least loaded group with room.  The pattern of an arrived request is
        analysed on a helper thread and stream while steps run (up to
        `lookahead` requests ahead), so admission costs no analysis."""
        import concurrent.futures
        import threading
        import torch
        engines = self._engine()
        reqs = sorted(requests, key=lambda r: r.arrival)
        # the producer hands over each update in pinned host memory
        host = {r.rid: [(_pinned(v), _pinned(b)) for v, b in r.updates] for r in reqs}
        xout = {r.rid: torch.empty((r.n, 4), dtype=torch.float64).pin_memory() for r in reqs}
        lock = threading.Lock()
        st = {"queue": collections.deque(reqs), "analysed": {}, "pat_used": 0.0,
              "load": [0] * self.groups, "active": [0] * self.groups}
        results = {}
        errors = []
        opts = dict(restart=self.restart, rtol=self.rtol, build_sweeps=self.build_sweeps,
                    apply_sweeps_lower=self.apply_sweeps, apply_sweeps_upper=self.apply_sweeps,
                    mode=self.mode)
        helper = concurrent.futures.ThreadPoolExecutor(max_workers=1)
        hstream = torch.cuda.Stream()
        dev = torch.cuda.current_device()

        def analyse(r):
            torch.cuda.set_device(dev)
            with torch.cuda.stream(hstream):
                rp = torch.from_numpy(r.rowptr).cuda()
                ci = torch.from_numpy(r.colind).cuda()
                return ab.Pattern(rp, ci, stream=hstream)

        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def admit(g, eng, active):
            """Under the lock: analyses ahead, then admissions into group g."""
            t = now()
            q, an = st["queue"], st["analysed"]
            for r in list(q)[:lookahead]:
                if r.arrival > t:
                    break
                pb = pattern_bytes(r.n, r.nnzb)
                if r.rid not in an and (st["pat_used"] + pb <= self.pattern_budget
                                        or (not an and not any(st["active"]))):
                    an[r.rid] = helper.submit(analyse, r)
                    st["pat_used"] += pb
            while q and q[0].arrival <= t and q[0].rid in an:
                r = q[0]
                fut = an[r.rid]
                if not fut.done():
                    if active:
                        break              # its analysis still runs: this group steps first
                    fut.result()
                # the least loaded group with room takes it: this one only if
                # no other group has less work (the others try after their steps)
                if any(st["load"][h] < st["load"][g] for h in range(self.groups) if h != g) \
                        and active:
                    break
                sid = eng.add_pattern(fut.result())
                if sid is None:
                    if not active and not any(st["active"]):
                        raise ValueError(f"request {r.rid} ({r.n} cells) does not fit an arena "
                                         f"({self.cells} cells)")
                    break                  # no room here now
                q.popleft()
                del an[r.rid]
                st["load"][g] += r.n
                st["active"][g] += 1
                active.append({"r": r, "id": sid, "k": 0, "ready": r.arrival,
                               "pb": pattern_bytes(r.n, r.nnzb),
                               "res": RequestResult(r.rid, r.n, r.arrival, now(), 0.0)})

        def worker(g):
            try:
                torch.cuda.set_device(dev)
                eng = engines[g]
                gstream = torch.cuda.Stream()
                active = []
                while True:
                    with lock:
                        admit(g, eng, active)
                        if not active and not st["queue"]:
                            return
                    if not active:
                        time.sleep(0.0002)
                        continue
                    free, total = torch.cuda.mem_get_info()
                    with lock:
                        self.memory_samples.append((now(), total - free))
                    out = eng.step([a["id"] for a in active],
                                   [host[a["r"].rid][a["k"]][0] for a in active],
                                   [host[a["r"].rid][a["k"]][1] for a in active],
                                   [xout[a["r"].rid] for a in active], stream=gstream, **opts)
                    tend = now()
                    k = len(active)
                    still = []
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
                        if a["k"] == len(a["r"].updates):
                            eng.remove(a["id"])
                            res.finished = tend
                            with lock:
                                st["pat_used"] -= a["pb"]
                                st["load"][g] -= a["r"].n
                                st["active"][g] -= 1
                                results[a["r"].rid] = res
                        else:
                            still.append(a)
                    active = still
            except Exception as e:   # surfaced after the run
                errors.append(e)
                with lock:
                    st["queue"].clear()

        threads = [threading.Thread(target=worker, args=(g,), daemon=True)
                   for g in range(self.groups)]
        try:
            for th in threads:
                th.start()
            for th in threads:
                th.join()
        finally:
            helper.shutdown(wait=True)
        if errors:
            raise errors[0]
        wall = now()
        return [results[r.rid] for r in requests], wall

    def close(self):
        self.engines = None


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
