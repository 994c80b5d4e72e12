"""Thin Python binding of libabilu (the C ABI in include/abilu.h).

Argument marshalling only: torch tensors supply device memory and
``torch.cuda`` streams supply the stream handle; every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback:
if libabilu.so is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libabilu.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; "
                      "g.build()'` (needs nvcc)")

_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, WARN_SINGULAR = range(7)
STATUS_NAMES = {0: "ABILU_OK", 1: "ABILU_EINVAL", 2: "ABILU_ENOMEM", 3: "ABILU_ECUDA",
                4: "ABILU_ENOCONV", 5: "ABILU_ETIMEOUT", 6: "ABILU_WARN_SINGULAR"}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2}
MODES = {"sync": 0, "async": 1}
INITS = {"a": 0, "previous": 1}

# every symbol the header declares
EXPORTS = ("abilu_version", "abilu_last_error", "abilu_kernel_launches", "abilu_pattern_create", "abilu_pattern_destroy",
           "abilu_pattern_counts", "abilu_factors_create", "abilu_factors_destroy",
           "abilu_factors_create_scalar", "abilu_build",
           "abilu_apply", "bsr_spmv", "abilu_factors_export", "abilu_factors_status",
           "abilu_factors_timing", "abilu_factors_sweep_time", "abilu_factors_diagnostics",
           "fgmres_default_opts", "fgmres_solve", "abilu_apply_noalloc", "abilu_batch_create",
           "abilu_batch_destroy", "abilu_batch_counts", "abilu_batch_set_system",
           "abilu_batch_solve", "abilu_batch_get_solution", "abilu_order",
           "abilu_permute_pattern", "abilu_gather_blocks", "abilu_add_block_diagonal",
           "abilu_to_f32", "abilu_mg_default_opts", "abilu_mg_create", "abilu_mg_destroy",
           "abilu_mg_setup", "abilu_mg_apply", "abilu_mg_levels", "abilu_mg_level_data",
           "fgmres_solve_mg", "abilu_parilut_default_opts", "abilu_parilut",
           "abilu_pattern_arrays", "abilu_factors_inject_stall", "abilu_factors_set_spin_limit",
           "abilu_server_arena_bytes", "abilu_server_create", "abilu_server_destroy",
           "abilu_server_add", "abilu_server_remove", "abilu_server_step", "abilu_server_usage",
           "abilu_factors_set_build_chunk", "abilu_batch_set_build_chunk",
           "abilu_server_add_pattern")


class FgmresOpts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iters", C.c_int32), ("rtol", C.c_double),
                ("build_sweeps", C.c_int32), ("apply_sweeps_lower", C.c_int32),
                ("apply_sweeps_upper", C.c_int32), ("mode", C.c_int32), ("build", C.c_int32),
                ("init", C.c_int32), ("reorth", C.c_int32), ("zero_guess", C.c_int32),
                ("spin_limit", C.c_int64)]


class MgOpts(C.Structure):
    _fields_ = [("max_levels", C.c_int32), ("min_coarse", C.c_int32), ("theta", C.c_double),
                ("factor_dtype", C.c_int32), ("build_sweeps", C.c_int32),
                ("apply_sweeps_lower", C.c_int32), ("apply_sweeps_upper", C.c_int32),
                ("pre_smooth", C.c_int32), ("post_smooth", C.c_int32),
                ("coarse_smooth", C.c_int32), ("mode", C.c_int32), ("init", C.c_int32)]


MG_MAX_LEVELS = 16


class ParilutOpts(C.Structure):
    _fields_ = [("fill", C.c_double), ("iters", C.c_int32), ("sweeps", C.c_int32),
                ("factor_dtype", C.c_int32)]


class ServerOpts(C.Structure):
    _fields_ = [("max_cells", C.c_int64), ("max_blocks", C.c_int64), ("max_systems", C.c_int32),
                ("factor_dtype", C.c_int32), ("restart", C.c_int32), ("max_lower", C.c_int64),
                ("max_upper", C.c_int64), ("max_pairs", C.c_int64), ("max_work", C.c_int64)]


class FgmresResult(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("rel_resid_est", C.c_double),
                ("rel_resid_true", C.c_double), ("singular_blocks", C.c_int64),
                ("status", C.c_int32)]


_vp, _i32, _i64, _f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_lib.abilu_version.restype = C.c_char_p
_lib.abilu_last_error.restype = C.c_char_p
_lib.abilu_kernel_launches.restype = C.c_uint64
_lib.abilu_kernel_launches.argtypes = []
_lib.abilu_pattern_create.argtypes = [_i32, _i32, _vp, _vp, _vp, C.POINTER(_vp)]
_lib.abilu_pattern_destroy.argtypes = [_vp]
_lib.abilu_pattern_destroy.restype = None
_lib.abilu_pattern_counts.argtypes = [_vp, C.POINTER(_i64)]
_lib.abilu_factors_create.argtypes = [_vp, C.c_int, C.POINTER(_vp)]
_lib.abilu_factors_create_scalar.argtypes = [_vp, C.c_int, C.POINTER(_vp)]
_lib.abilu_factors_destroy.argtypes = [_vp]
_lib.abilu_factors_destroy.restype = None
_lib.abilu_build.argtypes = [_vp, _vp, C.c_int, C.c_int, C.c_int, _vp]
_lib.abilu_apply.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp]
_lib.bsr_spmv.argtypes = [_vp, _vp, _f64, _vp, _f64, _vp, _vp]
_lib.abilu_apply_noalloc.argtypes = [_i32, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, C.c_int, _vp]
_lib.abilu_to_f32.argtypes = [_vp, _vp, _i64, _vp]
_lib.abilu_add_block_diagonal.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.abilu_order.argtypes = [_i32, _vp, _vp, _vp, _vp, _i32, _f64, _vp, _vp]
_lib.abilu_permute_pattern.argtypes = [_i32, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.abilu_gather_blocks.argtypes = [_i64, _vp, _vp, _vp, _vp]
_lib.abilu_apply_noalloc.restype = C.c_int
_lib.abilu_factors_export.argtypes = [_vp, _vp, _vp, _vp]
_lib.abilu_factors_status.argtypes = [_vp, C.POINTER(_i64), _vp]
_lib.abilu_server_arena_bytes.argtypes = [C.POINTER(ServerOpts), C.POINTER(_i64)]
_lib.abilu_server_create.argtypes = [C.POINTER(ServerOpts), _vp, C.POINTER(_vp)]
_lib.abilu_server_destroy.argtypes = [_vp]
_lib.abilu_server_destroy.restype = None
_lib.abilu_server_add.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp, C.POINTER(_i32)]
_lib.abilu_server_remove.argtypes = [_vp, _i32]
_lib.abilu_server_add_pattern.argtypes = [_vp, _vp, C.POINTER(_i32)]
_lib.abilu_server_add_pattern.restype = C.c_int
_lib.abilu_server_step.argtypes = [_vp, _i32, C.POINTER(_i32), C.POINTER(_vp), C.POINTER(_vp),
                                   C.POINTER(_vp), C.POINTER(FgmresOpts), C.POINTER(FgmresResult),
                                   _vp]
_lib.abilu_server_usage.argtypes = [_vp, C.POINTER(_i64)]
for _nm in ("abilu_server_arena_bytes", "abilu_server_create", "abilu_server_add",
            "abilu_server_remove", "abilu_server_step", "abilu_server_usage"):
    getattr(_lib, _nm).restype = C.c_int
_lib.abilu_factors_set_build_chunk.argtypes = [_vp, _i32]
_lib.abilu_factors_set_build_chunk.restype = C.c_int
_lib.abilu_batch_set_build_chunk.argtypes = [_vp, _i32]
_lib.abilu_batch_set_build_chunk.restype = C.c_int
_lib.abilu_factors_set_spin_limit.argtypes = [_vp, _i64]
_lib.abilu_factors_set_spin_limit.restype = C.c_int
_lib.abilu_factors_inject_stall.argtypes = [_vp, C.c_int]
_lib.abilu_factors_inject_stall.restype = C.c_int
_lib.abilu_factors_timing.argtypes = [_vp, C.c_int]
_lib.abilu_factors_timing.restype = C.c_int
_lib.abilu_factors_sweep_time.argtypes = [_vp, C.POINTER(C.c_float)]
_lib.abilu_factors_sweep_time.restype = C.c_int
_lib.abilu_factors_diagnostics.argtypes = [_vp, _vp, C.POINTER(_f64), _vp]
_lib.abilu_factors_diagnostics.restype = C.c_int
_lib.fgmres_default_opts.argtypes = [C.POINTER(FgmresOpts)]
_lib.fgmres_default_opts.restype = None
_lib.fgmres_solve.argtypes = [_vp, _vp, _vp, _vp, _vp, C.POINTER(FgmresOpts),
                              C.POINTER(FgmresResult), _vp]
_lib.abilu_batch_create.argtypes = [_i32, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_vp),
                                   C.POINTER(_vp), C.c_int, _vp, C.POINTER(_vp)]
_lib.abilu_batch_destroy.argtypes = [_vp]
_lib.abilu_batch_destroy.restype = None
_lib.abilu_batch_counts.argtypes = [_vp, C.POINTER(_i64)]
_lib.abilu_batch_set_system.argtypes = [_vp, _i32, _vp, _vp, _vp]
_lib.abilu_batch_solve.argtypes = [_vp, C.POINTER(FgmresOpts), C.POINTER(FgmresResult), _vp]
_lib.abilu_batch_get_solution.argtypes = [_vp, _i32, _vp, _vp]
_lib.abilu_mg_default_opts.argtypes = [C.POINTER(MgOpts)]
_lib.abilu_mg_default_opts.restype = None
_lib.abilu_mg_create.argtypes = [_vp, _vp, C.POINTER(MgOpts), _vp, C.POINTER(_vp)]
_lib.abilu_mg_destroy.argtypes = [_vp]
_lib.abilu_mg_destroy.restype = None
_lib.abilu_mg_setup.argtypes = [_vp, _vp, _vp]
_lib.abilu_mg_apply.argtypes = [_vp, _vp, _vp, _vp]
_lib.abilu_mg_levels.argtypes = [_vp, C.POINTER(_i64)]
_lib.abilu_mg_level_data.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.fgmres_solve_mg.argtypes = [_vp, _vp, _vp, _vp, C.POINTER(FgmresOpts),
                                 C.POINTER(FgmresResult), _vp]
_lib.abilu_pattern_arrays.argtypes = [_vp, _vp, _vp, _vp]
_lib.abilu_pattern_arrays.restype = C.c_int
_lib.abilu_parilut_default_opts.argtypes = [C.POINTER(ParilutOpts)]
_lib.abilu_parilut_default_opts.restype = None
_lib.abilu_parilut.argtypes = [_vp, _vp, C.POINTER(ParilutOpts), _vp, C.POINTER(_vp),
                               C.POINTER(_vp)]
for _nm in ("abilu_mg_create", "abilu_mg_setup", "abilu_mg_apply", "abilu_mg_levels",
            "abilu_mg_level_data", "fgmres_solve_mg", "abilu_parilut"):
    getattr(_lib, _nm).restype = C.c_int
for _nm in ("abilu_batch_create", "abilu_batch_counts", "abilu_batch_set_system",
            "abilu_batch_solve", "abilu_batch_get_solution", "abilu_order",
           "abilu_permute_pattern", "abilu_gather_blocks", "abilu_add_block_diagonal",
           "abilu_to_f32"):
    getattr(_lib, _nm).restype = C.c_int
for _nm in ("abilu_pattern_create", "abilu_pattern_counts", "abilu_factors_create", "abilu_build",
            "abilu_apply", "bsr_spmv", "abilu_factors_export", "abilu_factors_status",
           "abilu_factors_diagnostics",
            "fgmres_solve"):
    getattr(_lib, _nm).restype = C.c_int


class AbiluError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def version() -> str:
    return _lib.abilu_version().decode()


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_lib.abilu_kernel_launches())


def _check(status, allow=(OK,)):
    if status not in allow:
        raise AbiluError(status, _lib.abilu_last_error().decode())
    return status


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t, dtype, numel=None, what="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} must have {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Pattern:
    """Analysed block pattern (abilu_pattern_create)."""

    def __init__(self, rowptr, colind, stream=None):
        import torch
        n = rowptr.numel() - 1
        nnzb = colind.numel()
        h = C.c_void_p()
        _check(_lib.abilu_pattern_create(n, nnzb, _ptr(rowptr, torch.int32, what="rowptr"),
                                         _ptr(colind, torch.int32, what="colind"),
                                         _stream(stream), C.byref(h)))
        self.handle = h
        self.n, self.nnzb = n, nnzb

    @classmethod
    def _wrap(cls, handle):
        """A Python object owning an existing pattern handle."""
        self = cls.__new__(cls)
        self.handle = handle
        c = self.counts()
        self.n, self.nnzb = c["n"], c["nnzb"]
        return self

    def counts(self) -> dict:
        out = (C.c_int64 * 7)()
        _check(_lib.abilu_pattern_counts(self.handle, out))
        return dict(zip(("n", "nnzb", "nl", "nu", "npairs", "max_row", "nwork"), list(out)))

    def arrays(self, stream=None):
        """(rowptr, colind) of the pattern as new int32 CUDA tensors."""
        import torch
        rp = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(self.nnzb, dtype=torch.int32, device="cuda")
        _check(_lib.abilu_pattern_arrays(self.handle, _ptr(rp, torch.int32), _ptr(ci, torch.int32),
                                         _stream(stream)))
        return rp, ci

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.abilu_pattern_destroy(h)
            self.handle = None


class Factors:
    """Factor storage of one pattern (abilu_factors_create)."""

    def __init__(self, pattern: Pattern, dtype: str = "f32", scalar: bool = False):
        """scalar=True: the scalar ILU(0) variant (abilu_factors_create_scalar, FP64)."""
        h = C.c_void_p()
        create = _lib.abilu_factors_create_scalar if scalar else _lib.abilu_factors_create
        _check(create(pattern.handle, DTYPES[dtype], C.byref(h)))
        self.handle = h
        self.pattern = pattern
        self.dtype = dtype
        self.scalar = bool(scalar)

    def build(self, A, nsweeps, mode="sync", init="a", stream=None):
        import torch
        _check(_lib.abilu_build(self.handle, _ptr(A, torch.float64, 16 * self.pattern.nnzb, "A"),
                                int(nsweeps), MODES[mode], INITS[init], _stream(stream)))

    def apply(self, r, z, nsweeps_lower, nsweeps_upper, mode="sync", stream=None):
        import torch
        nv = 4 * self.pattern.n
        _check(_lib.abilu_apply(self.handle, _ptr(r, torch.float64, nv, "r"),
                                _ptr(z, torch.float64, nv, "z"), int(nsweeps_lower),
                                int(nsweeps_upper), MODES[mode], _stream(stream)))

    def export(self, stream=None):
        import torch
        X = torch.empty((self.pattern.nnzb, 4, 4), dtype=torch.float64, device="cuda")
        D = torch.empty((self.pattern.n, 4, 4), dtype=torch.float64, device="cuda")
        _check(_lib.abilu_factors_export(self.handle, _ptr(X, torch.float64),
                                         _ptr(D, torch.float64), _stream(stream)))
        return X, D

    def diagnostics(self, A, stream=None) -> dict:
        """ILU fixed-point residual, LU defect and Jacobi-matrix norms (FP64)."""
        import torch
        out = (C.c_double * 4)()
        _check(_lib.abilu_factors_diagnostics(self.handle,
                                              _ptr(A, torch.float64, 16 * self.pattern.nnzb, "A"),
                                              out, _stream(stream)))
        return dict(zip(("ilu_residual_l1", "lu_defect_max", "jacobi_norm_L", "jacobi_norm_U"),
                        list(out)))

    def timing(self, enable: bool = True):
        """Record CUDA events around the sweep kernels of every later build
        (abilu_factors_timing); sweep_ms() reads the last one."""
        _check(_lib.abilu_factors_timing(self.handle, int(bool(enable))))

    def sweep_ms(self) -> float:
        """Device time of the last timed build's sweep kernels, in ms."""
        v = C.c_float()
        _check(_lib.abilu_factors_sweep_time(self.handle, C.byref(v)))
        return v.value

    def set_spin_limit(self, limit: int = 0):
        """Polls before a bounded device wait of this handle's direct builds
        and applications gives up (0: the library default)."""
        _check(_lib.abilu_factors_set_spin_limit(self.handle, int(limit)))

    def set_build_chunk(self, blocks: int = 0):
        """Work blocks per ticket of the asynchronous build (0: the default)."""
        _check(_lib.abilu_factors_set_build_chunk(self.handle, int(blocks)))

    def inject_stall(self, enable: bool = True):
        """Failure injection for tests of the bounded waits
        (abilu_factors_inject_stall): the next ordered asynchronous build's
        waits run out after the spin limit and report ABILU_ETIMEOUT."""
        _check(_lib.abilu_factors_inject_stall(self.handle, int(bool(enable))))

    def singular_blocks(self, stream=None) -> int:
        v = C.c_int64()
        _check(_lib.abilu_factors_status(self.handle, C.byref(v), _stream(stream)))
        return v.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.abilu_factors_destroy(h)
            self.handle = None


def bsr_spmv(pattern: Pattern, A, x, y, alpha=1.0, beta=0.0, stream=None):
    import torch
    nv = 4 * pattern.n
    _check(_lib.bsr_spmv(pattern.handle, _ptr(A, torch.float64, 16 * pattern.nnzb, "A"),
                         float(alpha), _ptr(x, torch.float64, nv, "x"), float(beta),
                         _ptr(y, torch.float64, nv, "y"), _stream(stream)))


ORDERINGS = {"rcm": 0, "1wd": 1, "line": 2, "line-rcm": 3, "line-1wd": 4}


def _host(a, dtype):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, C.c_void_p(a.ctypes.data)


def order(rowptr, colind, kind="rcm", weights=None, vals=None, line_threshold=10.0):
    """abilu_order on host (numpy) arrays: returns (perm, line_of), perm[k] =
    the old index of the cell numbered k, line_of[c] = the line of old cell c
    (-1: none)."""
    import numpy as np
    n = len(rowptr) - 1
    rp, prp = _host(rowptr, np.int32)
    ci, pci = _host(colind, np.int32)
    w, pw = _host(weights, np.float64) if weights is not None else (None, None)
    v, pv = _host(vals, np.float64) if vals is not None else (None, None)
    perm = np.empty(n, np.int32)
    line_of = np.empty(n, np.int32)
    _check(_lib.abilu_order(n, prp, pci, pw, pv, ORDERINGS[kind], float(line_threshold),
                            C.c_void_p(perm.ctypes.data), C.c_void_p(line_of.ctypes.data)))
    return perm, line_of


def permute_pattern(rowptr, colind, perm):
    """abilu_permute_pattern on host arrays: (rowptr, colind, src) of the
    pattern renumbered by perm; src[p] = the old position of new block p."""
    import numpy as np
    n = len(rowptr) - 1
    rp, prp = _host(rowptr, np.int32)
    ci, pci = _host(colind, np.int32)
    pm, ppm = _host(perm, np.int32)
    ro = np.empty(n + 1, np.int32)
    co = np.empty(len(colind), np.int32)
    src = np.empty(len(colind), np.int32)
    _check(_lib.abilu_permute_pattern(n, prp, pci, ppm, C.c_void_p(ro.ctypes.data),
                                      C.c_void_p(co.ctypes.data), C.c_void_p(src.ctypes.data)))
    return ro, co, src


def gather_blocks(src, vals_in, vals_out, stream=None):
    """abilu_gather_blocks: vals_out[p] = vals_in[src[p]] on the device."""
    import torch
    nnzb = src.numel()
    _check(_lib.abilu_gather_blocks(nnzb, _ptr(src, torch.int32, what="src"),
                                    _ptr(vals_in, torch.float64, what="vals_in"),
                                    _ptr(vals_out, torch.float64, 16 * nnzb, "vals_out"),
                                    _stream(stream)))


def add_block_diagonal(pattern: Pattern, A_in, A_out, d, stream=None):
    """abilu_add_block_diagonal: A_out = A_in + diag(d_i) on the diagonal blocks
    (the pseudo-time shift of Sec. 2); A_in and A_out may be the same tensor."""
    import torch
    nb = 16 * pattern.nnzb
    _check(_lib.abilu_add_block_diagonal(pattern.handle, _ptr(A_in, torch.float64, nb, "A_in"),
                                         _ptr(A_out, torch.float64, nb, "A_out"),
                                         _ptr(d, torch.float64, 4 * pattern.n, "d"), _stream(stream)))


def to_f32(x, out, stream=None):
    """abilu_to_f32: FP64 -> FP32 round to nearest even with integer
    instructions (the conversion of the FGMRES normalisation)."""
    import torch
    _check(_lib.abilu_to_f32(_ptr(x, torch.float64, what="x"),
                             _ptr(out, torch.float32, x.numel(), "out"), x.numel(), _stream(stream)))


NOALLOC_MAX_CELLS = 65536


def apply_noalloc(rowptr, colind, X, Dinv, r, z, nsweeps_lower, nsweeps_upper, stream=None):
    """abilu_apply_noalloc: synchronous FP64 application on factors given as
    arrays (A's pattern layout), with no device allocation by the library."""
    import torch
    n = rowptr.numel() - 1
    _check(_lib.abilu_apply_noalloc(n, _ptr(rowptr, torch.int32, what="rowptr"),
                                    _ptr(colind, torch.int32, what="colind"),
                                    _ptr(X, torch.float64, 16 * colind.numel(), "X"),
                                    _ptr(Dinv, torch.float64, 16 * n, "Dinv"),
                                    _ptr(r, torch.float64, 4 * n, "r"),
                                    _ptr(z, torch.float64, 4 * n, "z"), int(nsweeps_lower),
                                    int(nsweeps_upper), _stream(stream)))


@dataclass
class SolveResult:
    iters: int
    restarts: int
    rel_resid_est: float
    rel_resid_true: float
    singular_blocks: int
    status: int

    @property
    def converged(self) -> bool:
        return self.status in (OK, WARN_SINGULAR)


def default_opts() -> FgmresOpts:
    o = FgmresOpts()
    _lib.fgmres_default_opts(C.byref(o))
    return o


def fgmres_solve(pattern: Pattern, A, factors: Factors, b, x, restart=30, max_iters=2500,
                 rtol=1e-6, build_sweeps=1, apply_sweeps_lower=3, apply_sweeps_upper=3,
                 mode="async", build=True, init="a", reorth=False, stream=None,
                 raise_on_noconv=False, zero_guess=False, spin_limit=0) -> SolveResult:
    import torch
    o = FgmresOpts(int(restart), int(max_iters), float(rtol), int(build_sweeps),
                   int(apply_sweeps_lower), int(apply_sweeps_upper), MODES[mode], int(bool(build)),
                   INITS[init], int(bool(reorth)), int(bool(zero_guess)), int(spin_limit))
    r = FgmresResult()
    nv = 4 * pattern.n
    st = _lib.fgmres_solve(pattern.handle, _ptr(A, torch.float64, 16 * pattern.nnzb, "A"),
                           factors.handle, _ptr(b, torch.float64, nv, "b"),
                           _ptr(x, torch.float64, nv, "x"), C.byref(o), C.byref(r),
                           _stream(stream))
    _check(st, allow=(OK, WARN_SINGULAR) if raise_on_noconv else (OK, WARN_SINGULAR, ENOCONV))
    return SolveResult(r.iters, r.restarts, r.rel_resid_est, r.rel_resid_true,
                       r.singular_blocks, st)


def _opts(restart, max_iters, rtol, build_sweeps, apply_sweeps_lower, apply_sweeps_upper, mode,
          build, init, reorth):
    return FgmresOpts(int(restart), int(max_iters), float(rtol), int(build_sweeps),
                      int(apply_sweeps_lower), int(apply_sweeps_upper), MODES[mode],
                      int(bool(build)), INITS[init], int(bool(reorth)), 1)


class Batch:
    """Many independent systems solved by the same launches (abilu_batch_*)."""

    def __init__(self, patterns, dtype="f32", stream=None):
        """patterns: list of (rowptr, colind) int32 CUDA tensors, one per system."""
        import torch
        nsys = len(patterns)
        self.n = [int(rp.numel() - 1) for rp, _ in patterns]
        self.nnzb = [int(ci.numel()) for _, ci in patterns]
        n_arr = (C.c_int32 * nsys)(*self.n)
        nz_arr = (C.c_int32 * nsys)(*self.nnzb)
        rps = (C.c_void_p * nsys)(*[_ptr(rp, torch.int32, what="rowptr").value for rp, _ in patterns])
        cis = (C.c_void_p * nsys)(*[_ptr(ci, torch.int32, what="colind").value for _, ci in patterns])
        h = C.c_void_p()
        _check(_lib.abilu_batch_create(nsys, n_arr, nz_arr, rps, cis, DTYPES[dtype],
                                       _stream(stream), C.byref(h)))
        self.handle = h
        self.nsys = nsys
        self.dtype = dtype

    def counts(self) -> dict:
        out = (C.c_int64 * 4)()
        _check(_lib.abilu_batch_counts(self.handle, out))
        return dict(zip(("nsys", "rows", "blocks", "chunks"), list(out)))

    def set_build_chunk(self, blocks: int = 0):
        """Work blocks per ticket of the batch's asynchronous build (0: default)."""
        _check(_lib.abilu_batch_set_build_chunk(self.handle, int(blocks)))

    def set_system(self, s, A=None, b=None, stream=None):
        import torch
        pa = _ptr(A, torch.float64, 16 * self.nnzb[s], "A") if A is not None else None
        pb = _ptr(b, torch.float64, 4 * self.n[s], "b") if b is not None else None
        _check(_lib.abilu_batch_set_system(self.handle, int(s), pa, pb, _stream(stream)))

    def solve(self, restart=30, max_iters=2500, rtol=1e-6, build_sweeps=1, apply_sweeps_lower=3,
              apply_sweeps_upper=3, mode="async", build=True, init="a", reorth=False,
              stream=None):
        o = _opts(restart, max_iters, rtol, build_sweeps, apply_sweeps_lower, apply_sweeps_upper,
                  mode, build, init, reorth)
        res = (FgmresResult * self.nsys)()
        st = _lib.abilu_batch_solve(self.handle, C.byref(o), res, _stream(stream))
        _check(st, allow=(OK, WARN_SINGULAR, ENOCONV))
        return [SolveResult(r.iters, r.restarts, r.rel_resid_est, r.rel_resid_true,
                            r.singular_blocks, r.status) for r in res]

    def solution(self, s, x, stream=None):
        import torch
        _check(_lib.abilu_batch_get_solution(self.handle, int(s),
                                             _ptr(x, torch.float64, 4 * self.n[s], "x"),
                                             _stream(stream)))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.abilu_batch_destroy(h)
            self.handle = None


def _server_opts(max_cells, max_blocks, max_systems, dtype, restart, max_lower=0, max_upper=0,
                 max_pairs=0, max_work=0):
    return ServerOpts(int(max_cells), int(max_blocks), int(max_systems), DTYPES[dtype],
                      int(restart), int(max_lower), int(max_upper), int(max_pairs), int(max_work))


def server_arena_bytes(max_cells, max_blocks, max_systems=64, dtype="f32", restart=30, **caps):
    """Device bytes of a server arena with these capacities (no device work)."""
    v = C.c_int64()
    o = _server_opts(max_cells, max_blocks, max_systems, dtype, restart, **caps)
    _check(_lib.abilu_server_arena_bytes(C.byref(o), C.byref(v)))
    return v.value


class NativeServer:
    """Continuous batching (abilu_server_*): every step solves one value update
    of each admitted system in shared launches; systems join and leave between
    steps inside one preallocated arena."""

    def __init__(self, max_cells, max_blocks, max_systems=64, dtype="f32", restart=30,
                 stream=None, **caps):
        o = _server_opts(max_cells, max_blocks, max_systems, dtype, restart, **caps)
        h = C.c_void_p()
        _check(_lib.abilu_server_create(C.byref(o), _stream(stream), C.byref(h)))
        self.handle = h
        self.dtype = dtype
        self.restart = int(restart)

    def add(self, rowptr, colind, stream=None):
        """Admit a system (device int32 rowptr/colind); returns its id, or None
        when the arena has no room for it now."""
        import torch
        n = rowptr.numel() - 1
        v = C.c_int32()
        st = _lib.abilu_server_add(self.handle, n, colind.numel(),
                                   _ptr(rowptr, torch.int32, what="rowptr"),
                                   _ptr(colind, torch.int32, what="colind"), _stream(stream),
                                   C.byref(v))
        if st == ENOMEM:
            return None
        _check(st)
        return v.value

    def add_pattern(self, pattern):
        """Admit a pattern analysed beforehand (a Pattern, e.g. made on another
        thread and stream); the server takes the handle over.  Returns the
        id, or None when the arena has no room for it now (the caller keeps
        the Pattern)."""
        v = C.c_int32()
        st = _lib.abilu_server_add_pattern(self.handle, pattern.handle, C.byref(v))
        if st == ENOMEM:
            return None
        _check(st)
        pattern.handle = None          # owned by the server now
        return v.value

    def remove(self, sid):
        _check(_lib.abilu_server_remove(self.handle, int(sid)))

    def usage(self) -> dict:
        out = (C.c_int64 * 14)()
        _check(_lib.abilu_server_usage(self.handle, out))
        names = ("rows", "blocks", "lower", "upper", "pairs", "work", "systems")
        return {"capacity": dict(zip(names, list(out)[:7])), "used": dict(zip(names, list(out)[7:]))}

    def step(self, ids, A, b, x, restart=30, max_iters=2500, rtol=1e-6, build_sweeps=1,
             apply_sweeps_lower=3, apply_sweeps_upper=3, mode="async", reorth=False, stream=None,
             spin_limit=0):
        """One batched solve of one update of every admitted system: ids, and
        per system A (nnzb,4,4), b and x (n,4) float64 tensors on the device or
        in pinned host memory."""
        k = len(ids)
        o = FgmresOpts(int(restart), int(max_iters), float(rtol), int(build_sweeps),
                       int(apply_sweeps_lower), int(apply_sweeps_upper), MODES[mode], 1, 0,
                       int(bool(reorth)), 1, int(spin_limit))
        for t in list(A) + list(b) + list(x):
            if not t.is_contiguous() or t.dtype.itemsize != 8:
                raise TypeError("server step arrays must be contiguous float64")
        idv = (C.c_int32 * k)(*[int(i) for i in ids])
        pa = (C.c_void_p * k)(*[t.data_ptr() for t in A])
        pb = (C.c_void_p * k)(*[t.data_ptr() for t in b])
        px = (C.c_void_p * k)(*[t.data_ptr() for t in x])
        res = (FgmresResult * k)()
        st = _lib.abilu_server_step(self.handle, k, idv, pa, pb, px, C.byref(o), res,
                                    _stream(stream))
        _check(st, allow=(OK, WARN_SINGULAR, ENOCONV))
        return [SolveResult(r.iters, r.restarts, r.rel_resid_est, r.rel_resid_true,
                            r.singular_blocks, r.status) for r in res]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.abilu_server_destroy(h)
            self.handle = None


class Multigrid:
    """V-cycle with block ILU smoothing on an aggregation hierarchy (abilu_mg_*)."""

    def __init__(self, pattern: Pattern, A, max_levels=10, min_coarse=512, theta=0.25,
                 factor_dtype="f32", build_sweeps=4, apply_sweeps_lower=2, apply_sweeps_upper=2,
                 pre_smooth=1, post_smooth=1, coarse_smooth=2, mode="sync", init="a",
                 stream=None):
        import torch
        o = MgOpts(int(max_levels), int(min_coarse), float(theta), DTYPES[factor_dtype],
                   int(build_sweeps), int(apply_sweeps_lower), int(apply_sweeps_upper),
                   int(pre_smooth), int(post_smooth), int(coarse_smooth), MODES[mode], INITS[init])
        h = C.c_void_p()
        _check(_lib.abilu_mg_create(pattern.handle, _ptr(A, torch.float64, 16 * pattern.nnzb, "A"),
                                    C.byref(o), _stream(stream), C.byref(h)))
        self.handle = h
        self.pattern = pattern   # the handle keeps the pattern: keep it alive
        self.A = A               # the values of the last set-up
        out = (C.c_int64 * (2 * MG_MAX_LEVELS + 1))()
        _check(_lib.abilu_mg_levels(h, out))
        self.nlevels = int(out[0])
        self.cells = [int(out[1 + 2 * k]) for k in range(self.nlevels)]
        self.blocks = [int(out[2 + 2 * k]) for k in range(self.nlevels)]

    def setup(self, A, stream=None):
        import torch
        _check(_lib.abilu_mg_setup(self.handle, _ptr(A, torch.float64, 16 * self.pattern.nnzb, "A"),
                                   _stream(stream)))
        self.A = A

    def apply(self, r, z, stream=None):
        import torch
        nv = 4 * self.pattern.n
        _check(_lib.abilu_mg_apply(self.handle, _ptr(r, torch.float64, nv, "r"),
                                   _ptr(z, torch.float64, nv, "z"), _stream(stream)))

    def level(self, k, factors=False, stream=None) -> dict:
        """Level k's aggregates (None on the coarsest), pattern and values, and
        with factors=True its block ILU factors in FP64 (X in the pattern
        layout, Dinv) - device tensors."""
        import torch
        n, nb = self.cells[k], self.blocks[k]
        agg = torch.empty(n, dtype=torch.int32, device="cuda") if k < self.nlevels - 1 else None
        rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(nb, dtype=torch.int32, device="cuda")
        v = torch.empty((nb, 4, 4), dtype=torch.float64, device="cuda")
        X = torch.empty((nb, 4, 4), dtype=torch.float64, device="cuda") if factors else None
        D = torch.empty((n, 4, 4), dtype=torch.float64, device="cuda") if factors else None
        _check(_lib.abilu_mg_level_data(self.handle, int(k),
                                        _ptr(agg, torch.int32) if agg is not None else None,
                                        _ptr(rp, torch.int32), _ptr(ci, torch.int32),
                                        _ptr(v, torch.float64),
                                        _ptr(X, torch.float64) if factors else None,
                                        _ptr(D, torch.float64) if factors else None,
                                        _stream(stream)))
        return dict(agg=agg, rowptr=rp, colind=ci, vals=v, X=X, Dinv=D)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.abilu_mg_destroy(h)
            self.handle = None


def fgmres_solve_mg(mg: Multigrid, A, b, x, restart=30, max_iters=2500, rtol=1e-6, build=True,
                    reorth=False, zero_guess=False, stream=None,
                    raise_on_noconv=False) -> SolveResult:
    """FGMRES right-preconditioned by one V-cycle per step (fgmres_solve_mg)."""
    import torch
    o = FgmresOpts(int(restart), int(max_iters), float(rtol), 0, 0, 0, 0, int(bool(build)), 0,
                   int(bool(reorth)), int(bool(zero_guess)))
    r = FgmresResult()
    nv = 4 * mg.pattern.n
    st = _lib.fgmres_solve_mg(mg.handle, _ptr(A, torch.float64, 16 * mg.pattern.nnzb, "A"),
                              _ptr(b, torch.float64, nv, "b"), _ptr(x, torch.float64, nv, "x"),
                              C.byref(o), C.byref(r), _stream(stream))
    _check(st, allow=(OK, WARN_SINGULAR) if raise_on_noconv else (OK, WARN_SINGULAR, ENOCONV))
    if build:
        mg.A = A
    return SolveResult(r.iters, r.restarts, r.rel_resid_est, r.rel_resid_true,
                       r.singular_blocks, st)


def parilut(pattern: Pattern, A, fill=2.0, iters=3, sweeps=2, dtype="f64", stream=None):
    """Threshold block ILU (abilu_parilut): (Pattern, Factors) of the final
    pattern, computed in FP64 and stored in `dtype`.  Use the factors with
    fgmres_solve(..., build=False)."""
    import torch
    o = ParilutOpts(float(fill), int(iters), int(sweeps), DTYPES[dtype])
    hp, hf = C.c_void_p(), C.c_void_p()
    _check(_lib.abilu_parilut(pattern.handle, _ptr(A, torch.float64, 16 * pattern.nnzb, "A"),
                              C.byref(o), _stream(stream), C.byref(hp), C.byref(hf)))
    pat = Pattern._wrap(hp)
    fac = Factors.__new__(Factors)
    fac.handle, fac.pattern, fac.dtype, fac.scalar = hf, pat, dtype, False
    return pat, fac
