"""CPU FP64 oracle for block ILU(0) by fixed-point sweeps, block triangular
sweeps, BSR SpMV and FGMRES.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this package; the CUDA library never imports, links or
calls it, and it imports nothing from the CUDA side.  The arithmetic lives in
``abilu_oracle.c`` (plain C, FP64, no FMA contraction); this module compiles it
with gcc on first use and wraps it with ctypes.  ``dense`` holds an independent
numpy brute force used to pin the C code.

Factor layout: X has A's pattern (L_ij at column < row, U_ij at column >= row),
Dinv holds inv(U_ii) per row.  Arrays are numpy: rowptr/colind int32,
A/X float64 (nnzb, 4, 4), Dinv float64 (n, 4, 4), vectors float64 (n, 4).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abilu_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "orderings.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_PI = C.POINTER(C.c_int32)
_PD = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f)
                                                for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Res(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("rel_resid_est", C.c_double), ("rel_resid_true", C.c_double)]


class _MgLevel(C.Structure):
    _fields_ = [("n", C.c_int32), ("rowptr", _PI), ("colind", _PI), ("A", _PD), ("X", _PD),
                ("Dinv", _PD), ("agg", _PI)]


class _Mg(C.Structure):
    _fields_ = [("nlevels", C.c_int), ("lv", C.POINTER(_MgLevel)), ("n_lower", C.c_int),
                ("n_upper", C.c_int), ("pre", C.c_int), ("post", C.c_int), ("coarse", C.c_int)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        i32, f64 = C.c_int32, C.c_double
        lib.orc_inv4.argtypes = [_PD, _PD]
        lib.orc_inv4.restype = C.c_int
        for nm in ("orc_bilu0_seq", "orc_bilu_init"):
            getattr(lib, nm).argtypes = [i32, _PI, _PI, _PD, _PD, _PD]
            getattr(lib, nm).restype = C.c_int
        lib.orc_bilu_sync_sweep.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD, _PD]
        lib.orc_bilu_sync_sweep.restype = C.c_int
        lib.orc_bilu_chunked_sweep.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, i32, _PI, i32]
        lib.orc_bilu_chunked_sweep.restype = C.c_int
        lib.orc_lower_sweep.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD]
        lib.orc_upper_sweep.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD, _PD]
        lib.orc_lower_solve.argtypes = [i32, _PI, _PI, _PD, _PD, _PD]
        lib.orc_upper_solve.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD]
        lib.orc_apply.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD, C.c_int, C.c_int, _PD]
        lib.orc_spmv.argtypes = [i32, _PI, _PI, _PD, _PD, _PD]
        lib.orc_fgmres.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, C.c_int, C.c_int, _PD, _PD,
                                   C.c_int, C.c_int, f64, C.POINTER(_Res), _PD]
        lib.orc_fgmres.restype = C.c_int
        lib.orc_ilu_residual_l1.argtypes = [i32, _PI, _PI, _PD, _PD, _PD]
        lib.orc_ilu_residual_l1.restype = f64
        lib.orc_lu_defect_max.argtypes = [i32, _PI, _PI, _PD, _PD]
        lib.orc_lu_defect_max.restype = f64
        lib.orc_jacobi_norms.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD]
        lib.orc_silu0_seq.argtypes = [i32, _PI, _PI, _PD, _PD]
        lib.orc_silu0_seq.restype = C.c_int
        lib.orc_silu_sync_sweep.argtypes = [i32, _PI, _PI, _PD, _PD, _PD]
        lib.orc_silu_sync_sweep.restype = C.c_int
        lib.orc_silu_lower_sweep.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD]
        lib.orc_silu_upper_sweep.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, _PD]
        lib.orc_silu_apply.argtypes = [i32, _PI, _PI, _PD, _PD, _PD, C.c_int, C.c_int, _PD]
        lib.orc_mg_aggregate.argtypes = [i32, _PI, _PI, _PD, f64, _PI]
        lib.orc_mg_aggregate.restype = i32
        lib.orc_galerkin_pattern.argtypes = [i32, _PI, _PI, _PI, i32, _PI, _PI]
        lib.orc_galerkin_pattern.restype = C.c_long
        lib.orc_galerkin_values.argtypes = [i32, _PI, _PI, _PD, _PI, i32, _PI, _PI, _PD]
        lib.orc_galerkin_values.restype = None
        lib.orc_mg_vcycle.argtypes = [C.POINTER(_Mg), _PD, _PD]
        lib.orc_mg_vcycle.restype = C.c_int
        lib.orc_fgmres_mg.argtypes = [C.POINTER(_Mg), _PD, _PD, C.c_int, C.c_int, f64,
                                      C.POINTER(_Res), _PD]
        lib.orc_fgmres_mg.restype = C.c_int
        lib.orc_fix_constant_upper.argtypes = [i32, _PI, _PI, _PD, _PD]
        lib.orc_fix_constant_upper.restype = None
        lib.orc_lu_pattern.argtypes = [i32, _PI, _PI, _PI, _PI]
        lib.orc_lu_pattern.restype = C.c_long
        lib.orc_keep_largest.argtypes = [C.c_long, _PD, C.c_long, C.POINTER(C.c_ubyte)]
        lib.orc_keep_largest.restype = C.c_long
        lib.orc_fgmres_ilu_pattern.argtypes = [i32, _PI, _PI, _PD, _PI, _PI, _PD, _PD, C.c_int,
                                               C.c_int, _PD, _PD, C.c_int, C.c_int, f64,
                                               C.POINTER(_Res), _PD]
        lib.orc_fgmres_ilu_pattern.restype = C.c_int
        lib.orc_order.argtypes = [i32, _PI, _PI, _PD, _PD, C.c_int, f64, _PI, _PI]
        lib.orc_order.restype = C.c_int
        for nm in ("orc_lower_sweep", "orc_upper_sweep", "orc_lower_solve", "orc_upper_solve",
                   "orc_apply", "orc_spmv", "orc_jacobi_norms", "orc_silu_lower_sweep",
                   "orc_silu_upper_sweep", "orc_silu_apply"):
            getattr(lib, nm).restype = None
        _lib = lib
    return _lib


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_PI)


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_PD)


def _pattern(rowptr, colind):
    rp, prp = _i(rowptr)
    ci, pci = _i(colind)
    return len(rp) - 1, (rp, ci), prp, pci


def inv4(a):
    """(inverse, singular flag) of one 4x4 block."""
    a, pa = _d(np.asarray(a, np.float64).reshape(4, 4))
    out = np.empty((4, 4))
    s = _load().orc_inv4(pa, out.ctypes.data_as(_PD))
    return out, bool(s)


def bilu0_seq(rowptr, colind, A):
    """Sequential block ILU(0) -> (X, Dinv, n_singular)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X = np.empty_like(A)
    Dinv = np.empty((n, 4, 4))
    s = _load().orc_bilu0_seq(n, prp, pci, pA, X.ctypes.data_as(_PD), Dinv.ctypes.data_as(_PD))
    return X, Dinv, s


def bilu_init(rowptr, colind, A):
    """Initial guess X^0 = A, Dinv^0 = inv(A_ii) -> (X, Dinv, n_singular)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X = np.empty_like(A)
    Dinv = np.empty((n, 4, 4))
    s = _load().orc_bilu_init(n, prp, pci, pA, X.ctypes.data_as(_PD), Dinv.ctypes.data_as(_PD))
    return X, Dinv, s


def bilu_sync_sweep(rowptr, colind, A, X, Dinv):
    """One synchronous sweep (X, Dinv) -> (X', Dinv', n_singular)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X, pX = _d(X)
    Dinv, pD = _d(Dinv)
    Xo = np.empty_like(X)
    Do = np.empty_like(Dinv)
    s = _load().orc_bilu_sync_sweep(n, prp, pci, pA, pX, pD, Xo.ctypes.data_as(_PD),
                                     Do.ctypes.data_as(_PD))
    return Xo, Do, s


def bilu_sync(rowptr, colind, A, nsweeps, X0=None, Dinv0=None):
    """``nsweeps`` synchronous sweeps from X^0 = A (or the given warm start)."""
    if X0 is None:
        X, Dinv, s = bilu_init(rowptr, colind, A)
    else:
        X, Dinv, s = np.array(X0, np.float64), np.array(Dinv0, np.float64), 0
    tot = s
    for _ in range(nsweeps):
        X, Dinv, s = bilu_sync_sweep(rowptr, colind, A, X, Dinv)
        tot += s
    return X, Dinv, tot


def bilu_chunked_sweep(rowptr, colind, A, X, Dinv, chunk, chunk_order):
    """In-place chunked sweep (deterministic emulation of the asynchronous one).
    X, Dinv are modified in place (they must be C-contiguous float64)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    assert X.dtype == np.float64 and X.flags.c_contiguous
    assert Dinv.dtype == np.float64 and Dinv.flags.c_contiguous
    co, pco = _i(chunk_order)
    return _load().orc_bilu_chunked_sweep(n, prp, pci, pA, X.ctypes.data_as(_PD),
                                          Dinv.ctypes.data_as(_PD), int(chunk), pco, len(co))


def lower_sweep(rowptr, colind, X, r, y_in):
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    r, pr = _d(r)
    y_in, py = _d(y_in)
    out = np.empty((n, 4))
    _load().orc_lower_sweep(n, prp, pci, pX, pr, py, out.ctypes.data_as(_PD))
    return out


def upper_sweep(rowptr, colind, X, Dinv, y, x_in):
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    Dinv, pD = _d(Dinv)
    y, py = _d(y)
    x_in, px = _d(x_in)
    out = np.empty((n, 4))
    _load().orc_upper_sweep(n, prp, pci, pX, pD, py, px, out.ctypes.data_as(_PD))
    return out


def lower_solve(rowptr, colind, X, r):
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    r, pr = _d(r)
    out = np.empty((n, 4))
    _load().orc_lower_solve(n, prp, pci, pX, pr, out.ctypes.data_as(_PD))
    return out


def upper_solve(rowptr, colind, X, Dinv, y):
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    Dinv, pD = _d(Dinv)
    y, py = _d(y)
    out = np.empty((n, 4))
    _load().orc_upper_solve(n, prp, pci, pX, pD, py, out.ctypes.data_as(_PD))
    return out


def apply(rowptr, colind, X, Dinv, r, n_lower, n_upper):
    """z ~= (LU)^{-1} r with the given sweep counts (negative: exact)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    Dinv, pD = _d(Dinv)
    r, pr = _d(r)
    z = np.empty((n, 4))
    work = np.empty(2 * n * 4)
    _load().orc_apply(n, prp, pci, pX, pD, pr, z.ctypes.data_as(_PD), int(n_lower),
                      int(n_upper), work.ctypes.data_as(_PD))
    return z


def spmv(rowptr, colind, A, x):
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    x, px = _d(x)
    y = np.empty((n, 4))
    _load().orc_spmv(n, prp, pci, pA, px, y.ctypes.data_as(_PD))
    return y


@dataclass
class FgmresResult:
    iters: int
    restarts: int
    converged: bool
    rel_resid_est: float
    rel_resid_true: float
    history: np.ndarray


def fgmres(rowptr, colind, A, X, Dinv, b, n_lower, n_upper, restart=30, max_iters=2500,
           rtol=1e-6, x0=None):
    """FGMRES(restart) with the block ILU preconditioner (X, Dinv) -> (x, result);
    Dinv=None: X holds scalar ILU factors (silu_*)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X, pX = _d(X)
    if Dinv is None:
        pD = None
    else:
        Dinv, pD = _d(Dinv)
    b, pb = _d(b)
    x = np.zeros((n, 4)) if x0 is None else np.array(x0, np.float64)
    res = _Res()
    hist = np.full(max_iters + 1, np.nan)
    _load().orc_fgmres(n, prp, pci, pA, pX, pD, int(n_lower), int(n_upper), pb,
                       x.ctypes.data_as(_PD), int(restart), int(max_iters), float(rtol),
                       C.byref(res), hist.ctypes.data_as(_PD))
    return x, FgmresResult(res.iters, res.restarts, bool(res.converged), res.rel_resid_est,
                           res.rel_resid_true, hist[: res.iters + 1])


def ilu_residual_l1(rowptr, colind, A, X):
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X, pX = _d(X)
    work = np.empty(len(keep[1]) * 16 + n * 16)
    return _load().orc_ilu_residual_l1(n, prp, pci, pA, pX, work.ctypes.data_as(_PD))


def lu_defect_max(rowptr, colind, A, X):
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X, pX = _d(X)
    return _load().orc_lu_defect_max(n, prp, pci, pA, pX)


def jacobi_norms(rowptr, colind, X, Dinv):
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    Dinv, pD = _d(Dinv)
    ln, un = C.c_double(), C.c_double()
    _load().orc_jacobi_norms(n, prp, pci, pX, pD, C.byref(ln), C.byref(un))
    return ln.value, un.value


# ---------------------------------------------------------- scalar ILU(0)
# Factors in A's block layout: blocks left of the diagonal hold L entries,
# right of it U entries; a diagonal block holds its strictly lower L entries
# (unit diagonal implied) and the rest of U.

def silu0_seq(rowptr, colind, A):
    """Sequential scalar ILU(0) on the scalar pattern -> (X, replaced pivots)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X = np.empty_like(A)
    ns = _load().orc_silu0_seq(n, prp, pci, pA, X.ctypes.data_as(_PD))
    return X, ns


def silu_sync(rowptr, colind, A, nsweeps, X0=None):
    """nsweeps Chow-Patel Jacobi-type sweeps from X0 (default A) -> (X, replaced pivots)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X = np.array(A if X0 is None else X0, np.float64)
    Y = np.empty_like(X)
    total = 0
    for _ in range(nsweeps):
        total += _load().orc_silu_sync_sweep(n, prp, pci, pA, X.ctypes.data_as(_PD),
                                             Y.ctypes.data_as(_PD))
        X, Y = Y, X
    return X, total


def silu_lower_sweep(rowptr, colind, X, r, y_in):
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    r, pr = _d(r)
    y_in, py = _d(y_in)
    out = np.empty((n, 4))
    _load().orc_silu_lower_sweep(n, prp, pci, pX, pr, py, out.ctypes.data_as(_PD))
    return out


def silu_upper_sweep(rowptr, colind, X, y, x_in):
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    y, py = _d(y)
    x_in, px = _d(x_in)
    out = np.empty((n, 4))
    _load().orc_silu_upper_sweep(n, prp, pci, pX, py, px, out.ctypes.data_as(_PD))
    return out


def silu_apply(rowptr, colind, X, r, n_lower, n_upper):
    """z ~= (LU)^{-1} r with scalar factors (negative sweep counts: exact)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    X, pX = _d(X)
    r, pr = _d(r)
    z = np.empty((n, 4))
    work = np.empty(2 * n * 4)
    _load().orc_silu_apply(n, prp, pci, pX, pr, z.ctypes.data_as(_PD), int(n_lower),
                           int(n_upper), work.ctypes.data_as(_PD))
    return z


# ------------------------------------------------- multigrid smoother (f4)
# Block ILU sweeps as the smoother of an aggregation multigrid V-cycle: the
# paper names this as future work without fixing a cycle; the cycle here is the
# one the library implements (see abilu_oracle.c, "multigrid smoother").

def mg_aggregate(rowptr, colind, A, theta):
    """Greedy strong-coupling aggregation -> (agg int32[n], number of aggregates)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    agg = np.empty(n, np.int32)
    nc = _load().orc_mg_aggregate(n, prp, pci, pA, float(theta), agg.ctypes.data_as(_PI))
    if nc < 0:
        raise MemoryError("orc_mg_aggregate")
    return agg, int(nc)


def galerkin(rowptr, colind, A, agg, nc):
    """A_c = P^T A P for piecewise-constant P -> (rowptr_c, colind_c, Ac)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    agg, pg = _i(agg)
    rpc = np.empty(nc + 1, np.int32)
    cic = np.empty(max(len(keep[1]), 1), np.int32)
    nnz = _load().orc_galerkin_pattern(n, prp, pci, pg, int(nc), rpc.ctypes.data_as(_PI),
                                       cic.ctypes.data_as(_PI))
    if nnz < 0:
        raise MemoryError("orc_galerkin_pattern")
    cic = np.ascontiguousarray(cic[:nnz])
    Ac = np.empty((nnz, 4, 4))
    _load().orc_galerkin_values(n, prp, pci, pA, pg, int(nc), rpc.ctypes.data_as(_PI),
                                cic.ctypes.data_as(_PI), Ac.ctypes.data_as(_PD))
    return rpc, cic, Ac


@dataclass
class MgLevel:
    rowptr: np.ndarray
    colind: np.ndarray
    A: np.ndarray
    X: np.ndarray
    Dinv: np.ndarray
    agg: np.ndarray | None    # each cell's aggregate on the next level (None: coarsest)


def mg_hierarchy(rowptr, colind, A, theta=0.25, max_levels=10, min_coarse=512,
                 build_sweeps=4):
    """Levels of the cycle: coarsen while fewer than max_levels levels exist and
    the last has more than min_coarse cells, stopping when aggregation no longer
    reduces the cell count; every level's block ILU from build_sweeps
    synchronous sweeps (from X^0 = A)."""
    rp = np.ascontiguousarray(rowptr, np.int32)
    ci = np.ascontiguousarray(colind, np.int32)
    Av = np.ascontiguousarray(A, np.float64)
    mats = [(rp, ci, Av)]
    aggs = []
    while len(mats) < max_levels and len(mats[-1][0]) - 1 > min_coarse:
        r, c, a = mats[-1]
        agg, nc = mg_aggregate(r, c, a, theta)
        if nc >= len(r) - 1:
            break
        aggs.append(agg)
        mats.append(galerkin(r, c, a, agg, nc))
    levels = []
    for k, (r, c, a) in enumerate(mats):
        X, D, _ = bilu_sync(r, c, a, build_sweeps)
        levels.append(MgLevel(r, c, a, X, D, aggs[k] if k < len(aggs) else None))
    return levels


def _mg_struct(levels, n_lower, n_upper, pre, post, coarse):
    arr = (_MgLevel * len(levels))()
    keep = []
    for k, L in enumerate(levels):
        rp, prp = _i(L.rowptr)
        ci, pci = _i(L.colind)
        A, pA = _d(L.A)
        X, pX = _d(L.X)
        D, pD = _d(L.Dinv)
        if L.agg is not None:
            ag, pg = _i(L.agg)
            keep.append(ag)
        else:
            pg = None
        keep += [rp, ci, A, X, D]
        arr[k] = _MgLevel(len(rp) - 1, prp, pci, pA, pX, pD, pg)
    mg = _Mg(len(levels), arr, int(n_lower), int(n_upper), int(pre), int(post), int(coarse))
    return mg, (arr, keep)


def mg_vcycle(levels, r, n_lower, n_upper, pre=1, post=1, coarse=2):
    """z = one V-cycle applied to r, from zero (the multigrid preconditioner)."""
    mg, keep = _mg_struct(levels, n_lower, n_upper, pre, post, coarse)
    r, pr = _d(r)
    z = np.empty((len(levels[0].rowptr) - 1, 4))
    if _load().orc_mg_vcycle(C.byref(mg), pr, z.ctypes.data_as(_PD)) != 0:
        raise MemoryError("orc_mg_vcycle")
    return z


def fgmres_mg(levels, b, n_lower, n_upper, pre=1, post=1, coarse=2, restart=30,
              max_iters=2500, rtol=1e-6):
    """FGMRES(restart) right-preconditioned by one V-cycle -> (x, result)."""
    mg, keep = _mg_struct(levels, n_lower, n_upper, pre, post, coarse)
    b, pb = _d(b)
    x = np.zeros((len(levels[0].rowptr) - 1, 4))
    res = _Res()
    hist = np.full(max_iters + 1, np.nan)
    _load().orc_fgmres_mg(C.byref(mg), pb, x.ctypes.data_as(_PD), int(restart), int(max_iters),
                          float(rtol), C.byref(res), hist.ctypes.data_as(_PD))
    return x, FgmresResult(res.iters, res.restarts, bool(res.converged), res.rel_resid_est,
                           res.rel_resid_true, hist[: res.iters + 1])


# ------------------------------------------------- threshold block ILU (f4)
# A threshold block ILU by fixed-point sweeps, the extension the paper names
# last (parallel threshold ILU, ParILUT): the pattern grows by the fill of L U
# and is cut back to the largest blocks, with one synchronous sweep after each
# change.  The paper gives no algorithm; this is the library's reading.

def lu_pattern(rowptr, colind):
    """Block pattern of L U (L unit lower, U upper, both on the given pattern)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    rpo = np.empty(n + 1, np.int32)
    nnz = _load().orc_lu_pattern(n, prp, pci, rpo.ctypes.data_as(_PI), None)
    if nnz < 0:
        raise MemoryError("orc_lu_pattern")
    cio = np.empty(max(nnz, 1), np.int32)
    _load().orc_lu_pattern(n, prp, pci, rpo.ctypes.data_as(_PI), cio.ctypes.data_as(_PI))
    return rpo, np.ascontiguousarray(cio[:nnz])


def keep_largest(key, budget):
    """Mask of the entries above the (budget+1)-th largest key (all if <= budget)."""
    key, pk = _d(key)
    keep = np.empty(len(key), np.uint8)
    _load().orc_keep_largest(len(key), pk, int(budget), keep.ctypes.data_as(C.POINTER(C.c_ubyte)))
    return keep.astype(bool)


def block_norm2(vals):
    """Squared Frobenius norm of each block, entries summed in storage order."""
    v = np.asarray(vals, np.float64).reshape(-1, 16)
    s = np.zeros(len(v))
    for e in range(16):
        s = s + v[:, e] * v[:, e]
    return s


def fix_constant_upper(rowptr, colind, A, X):
    """Copy of X with every strictly upper block that has no product pair set
    to A's block (its update is constant; a build sets it before sweeping)."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    A, pA = _d(A)
    X = np.array(X, np.float64)
    _load().orc_fix_constant_upper(n, prp, pci, pA, X.ctypes.data_as(_PD))
    return X


def map_blocks(rowptr, colind, vals, rowptr_new, colind_new):
    """Blocks of `vals` (on rowptr/colind) placed on the new pattern, zero where absent."""
    n = len(rowptr) - 1
    key = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr)) * n + colind
    key_new = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr_new)) * n + colind_new
    pos = np.searchsorted(key, key_new)
    pos = np.minimum(pos, max(len(key) - 1, 0))
    found = (len(key) > 0) & (key[pos] == key_new)
    out = np.zeros((len(colind_new), 4, 4))
    out[found] = np.asarray(vals).reshape(-1, 4, 4)[pos[found]]
    return out


def parilut(rowptr, colind, A, fill=2.0, iters=3, sweeps=2):
    """Threshold block ILU -> (rowptr, colind, X, Dinv) on its final pattern.

    Budgets: floor(fill * blocks) strictly lower and strictly upper blocks, the
    block counts of A's pattern.  Start: X^0 = A, `sweeps` synchronous sweeps
    on A's pattern.  Then `iters` times: (1) the pattern becomes that of L U
    (which contains it), new blocks start at zero, A is taken as zero outside
    its own pattern, `sweeps` synchronous sweeps; (2) of the strictly lower
    blocks keep those whose squared norm exceeds the (budget+1)-th largest,
    likewise upper (diagonal blocks always), `sweeps` synchronous sweeps on the
    kept pattern.  Before the sweeps on a new pattern, its strictly upper
    blocks without product pairs take A's value (fix_constant_upper)."""
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    colind = np.ascontiguousarray(colind, np.int32)
    A = np.ascontiguousarray(A, np.float64)
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    budget_l = int(np.floor(fill * np.sum(rows > colind)))
    budget_u = int(np.floor(fill * np.sum(rows < colind)))
    X, D, _ = bilu_sync(rowptr, colind, A, sweeps)
    rp, ci = rowptr, colind
    for _ in range(iters):
        rp2, ci2 = lu_pattern(rp, ci)
        X2 = map_blocks(rp, ci, X, rp2, ci2)
        A2 = map_blocks(rowptr, colind, A, rp2, ci2)
        X2 = fix_constant_upper(rp2, ci2, A2, X2)
        for _ in range(sweeps):
            X2, D, _ = bilu_sync_sweep(rp2, ci2, A2, X2, D)
        r2 = np.repeat(np.arange(n), np.diff(rp2))
        key = block_norm2(X2)
        keep = r2 == ci2
        low, up = r2 > ci2, r2 < ci2
        keep[low] = keep_largest(key[low], budget_l)
        keep[up] = keep_largest(key[up], budget_u)
        ci = np.ascontiguousarray(ci2[keep])
        rp = np.concatenate([[0], np.cumsum(np.bincount(r2[keep], minlength=n))]).astype(np.int32)
        X, As = X2[keep], A2[keep]
        X = fix_constant_upper(rp, ci, As, X)
        for _ in range(sweeps):
            X, D, _ = bilu_sync_sweep(rp, ci, As, X, D)
    return rp, ci, X, D


def fgmres_ilu_pattern(rowptr, colind, A, rowptr_f, colind_f, X, Dinv, b, n_lower, n_upper,
                       restart=30, max_iters=2500, rtol=1e-6):
    """FGMRES on A preconditioned by block ILU factors on their own pattern."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    _, keepf, prf, pcf = _pattern(rowptr_f, colind_f)
    A, pA = _d(A)
    X, pX = _d(X)
    Dinv, pD = _d(Dinv)
    b, pb = _d(b)
    x = np.zeros((n, 4))
    res = _Res()
    hist = np.full(max_iters + 1, np.nan)
    _load().orc_fgmres_ilu_pattern(n, prp, pci, pA, prf, pcf, pX, pD, int(n_lower), int(n_upper),
                                   pb, x.ctypes.data_as(_PD), int(restart), int(max_iters),
                                   float(rtol), C.byref(res), hist.ctypes.data_as(_PD))
    return x, FgmresResult(res.iters, res.restarts, bool(res.converged), res.rel_resid_est,
                           res.rel_resid_true, hist[: res.iters + 1])


ORDERINGS = {"rcm": 0, "1wd": 1, "line": 2, "line-rcm": 3, "line-1wd": 4}


def order(rowptr, colind, kind="rcm", weights=None, vals=None, threshold=10.0):
    """Orderings of the cell graph (orderings.c; Sec. 5, 5.1, 5.2):
    (perm, line_of), perm[k] = the old index of the cell numbered k, line_of[c]
    = the line of cell c or -1."""
    n, keep, prp, pci = _pattern(rowptr, colind)
    pw = pv = None
    if weights is not None:
        w, pw = _d(weights)
    if vals is not None:
        v, pv = _d(vals)
    perm = np.empty(n, np.int32)
    line_of = np.empty(n, np.int32)
    rc = _load().orc_order(n, prp, pci, pw, pv, ORDERINGS[kind], float(threshold),
                           perm.ctypes.data_as(_PI), line_of.ctypes.data_as(_PI))
    if rc != 0:
        raise ValueError("orc_order: bad input")
    return perm, line_of
