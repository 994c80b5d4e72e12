"""Pseudo-time continuation driving the preconditioned linear solves (Sec. 2).

A steady problem r(w) = 0 is marched in pseudo-time with backward Euler
(Eq. pseudotimestep): every step solves

    (M_tau^n + dr/dw(w^n)) dw^n = -r(w^n),   w^{n+1} = w^n + omega dw^n,

where M_tau^n is block diagonal with blocks (V_i / dtau_i^n) I.  The local time
step comes from one CFL number for all cells, dtau_i = cfl * V_i / s_i (s_i the
sum over the cell's faces of the largest flux-Jacobian eigenvalue times the
face area), so the shift of row i is s_i / cfl.  The CFL number starts small and
is ramped by the ratio of successive residual norms (Eq. cfl): the exponent is
0.25 when the residual fell and 0.3 when it did not, and the value is kept
between the starting value and a maximum (10^4 in the paper's runs).

Each step is one linear solve on the same pattern with new values: FGMRES to a
relative drop of 0.1, at most 60 iterations, restart 30 (the paper's nonlinear
settings, Sec. 6), preconditioned by ABILU whose factors start from the
previous step's (the initial guess the paper allows for the factorisation in a
CFD simulation); the first step starts them from the matrix itself.  The
matrix of a step is assembled on the device: the caller's Jacobian values, then
the pseudo-time shift added to the diagonal blocks (abilu_add_block_diagonal).

The physics is the caller's: `residual(w, out)` writes r(w) and
`jacobian(w, out)` writes dr/dw on the pattern, both on the device.
`SemilinearProblem` is a model problem with that interface for tests and
benchmarks: r(w) = A w + kappa w |w| - f on a Jacobian-shaped block pattern.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

from . import abilu as _ab


def cfl_update(cfl: float, rnorm_old: float, rnorm_new: float, cfl_min: float,
               cfl_max: float) -> float:
    """Eq. (cfl): cfl * (||r^n|| / ||r^{n+1}||)^e with e = 0.25 if the ratio
    exceeds 1 and 0.3 otherwise, kept in [cfl_min, cfl_max]."""
    if rnorm_new <= 0.0:
        return cfl_max
    ratio = rnorm_old / rnorm_new
    e = 0.25 if ratio > 1.0 else 0.3
    return min(max(cfl * ratio ** e, cfl_min), cfl_max)


@dataclass
class Step:
    step: int
    cfl: float             # CFL number used in this step
    rnorm: float           # ||r(w^{n+1})||_2 after the step
    energy: float          # ||r_energy(w^{n+1})||_2 (the convergence measure)
    lin_iters: int
    lin_rel_resid: float   # true relative residual of the linear solve
    ms: float              # wall time of the step (host clock, synchronised)


class PseudoTimeSolver:
    def __init__(self, pattern: "_ab.Pattern", residual, jacobian, shift_scale, dtype="f32",
                 mode="async", cfl0=10.0, cfl_max=1e4, omega=1.0, lin_rtol=0.1,
                 lin_max_iters=60, restart=30, build_sweeps=1, apply_sweeps=3,
                 energy_component=3):
        import torch
        self.pattern = pattern
        self.residual, self.jacobian = residual, jacobian
        self.s = shift_scale                       # device double[n]: s_i (so M_tau,i = s_i / cfl)
        self.fac = _ab.Factors(pattern, dtype)
        self.mode = mode
        self.cfl0, self.cfl_max, self.omega = float(cfl0), float(cfl_max), float(omega)
        self.lin = dict(restart=restart, max_iters=lin_max_iters, rtol=lin_rtol,
                        build_sweeps=build_sweeps, apply_sweeps_lower=apply_sweeps,
                        apply_sweeps_upper=apply_sweeps, mode=mode)
        self.ec = energy_component
        n, nnzb = pattern.n, pattern.nnzb
        dev = shift_scale.device
        self.A = torch.empty((nnzb, 4, 4), dtype=torch.float64, device=dev)
        self.r = torch.empty((n, 4), dtype=torch.float64, device=dev)
        self.dw = torch.empty((n, 4), dtype=torch.float64, device=dev)
        self.d = torch.empty((n, 4), dtype=torch.float64, device=dev)

    def run(self, w, rel_tol=1e-6, max_steps=500):
        """March w (device double[n][4], updated in place) until the energy
        residual dropped by rel_tol; returns the list of Steps."""
        import torch
        self.residual(w, self.r)
        rn = float(torch.linalg.vector_norm(self.r))
        e0 = float(torch.linalg.vector_norm(self.r[:, self.ec]))
        cfl = self.cfl0
        log = []
        for n in range(max_steps):
            t0 = time.perf_counter()
            self.jacobian(w, self.A)
            self.d.copy_((self.s / cfl).unsqueeze(1).expand(-1, 4))
            _ab.add_block_diagonal(self.pattern, self.A, self.A, self.d)
            torch.neg(self.r, out=self.r)           # b = -r(w^n)
            res = _ab.fgmres_solve(self.pattern, self.A, self.fac, self.r, self.dw,
                                   init="a" if n == 0 else "previous", zero_guess=True,
                                   **self.lin)
            w.add_(self.dw, alpha=self.omega)
            self.residual(w, self.r)
            rn_new = float(torch.linalg.vector_norm(self.r))
            en = float(torch.linalg.vector_norm(self.r[:, self.ec]))
            torch.cuda.synchronize()
            log.append(Step(n, cfl, rn_new, en, res.iters, res.rel_resid_true,
                            (time.perf_counter() - t0) * 1e3))
            if not math.isfinite(rn_new):
                break
            cfl = cfl_update(cfl, rn, rn_new, self.cfl0, self.cfl_max)
            rn = rn_new
            if en <= rel_tol * e0:
                break
        return log


class SemilinearProblem:
    """r(w) = A w + kappa w|w| - f (componentwise w|w|) on a block pattern:
    dr/dw = A + diag(2 kappa |w|).  The residual uses the library's FP64 SpMV;
    the Jacobian adds 2 kappa |w_i| to the diagonal blocks of A."""

    def __init__(self, pattern: "_ab.Pattern", A, f, kappa: float):
        self.pattern, self.A, self.f, self.kappa = pattern, A, f, float(kappa)

    def residual(self, w, out):
        _ab.bsr_spmv(self.pattern, self.A, w, out)
        out.addcmul_(w, w.abs(), value=self.kappa).sub_(self.f)

    def jacobian(self, w, out):
        d = w.abs().mul_(2.0 * self.kappa)
        _ab.add_block_diagonal(self.pattern, self.A, out, d)
