"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a worked
example done by hand, numpy/scipy library routines, the dense IKJ brute force in
oracle/dense.py (written independently), closed forms for special structures,
and the paper's finite-convergence theorems (Sec. 4.1-4.2).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import abilu_inputs as gen
import oracle
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sys(nx=4, ny=3, seed=0, order="rcm", **kw):
    return gen.small_system(nx, ny, seed=seed, order=order, **kw)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _bsr(rowptr, colind, vals):
    n = len(rowptr) - 1
    return sp.bsr_matrix((np.asarray(vals), colind, rowptr), shape=(4 * n, 4 * n))


def _chain_depth(rowptr, colind, lower=True):
    """Longest chain of strictly decreasing (lower) / increasing (upper) neighbours."""
    n = len(rowptr) - 1
    depth = np.zeros(n, int)
    rng = range(n) if lower else range(n - 1, -1, -1)
    for i in rng:
        cols = colind[rowptr[i]:rowptr[i + 1]]
        ks = cols[cols < i] if lower else cols[cols > i]
        depth[i] = depth[ks].max() + 1 if len(ks) else 0
    return int(depth.max())


# ------------------------------------------------------------------ 4x4 inverse

def test_inv4_matches_numpy():
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = rng.standard_normal((4, 4)) + 3 * np.eye(4) * rng.choice([-1, 1])
        inv, sing = oracle.inv4(a)
        assert not sing
        assert _rel(inv, np.linalg.inv(a)) < 1e-13


def test_inv4_needs_pivoting():
    p = np.eye(4)[[2, 0, 3, 1]] * np.array([1.0, 2.0, 4.0, 8.0])
    inv, sing = oracle.inv4(p)
    assert not sing
    np.testing.assert_array_equal(inv, np.linalg.inv(p))


@pytest.mark.parametrize("a", [np.zeros((4, 4)), np.ones((4, 4)),
                               np.diag([1.0, 2.0, 0.0, 3.0]),
                               np.diag([1.0, np.nan, 1.0, 1.0])])
def test_inv4_singular_is_replaced_by_identity(a):
    inv, sing = oracle.inv4(a)
    assert sing
    np.testing.assert_array_equal(inv, np.eye(4))


# ------------------------------------------------------------ sequential BILU(0)

def _case(c):
    rowptr = np.array([0, 2, 4], np.int32)
    colind = np.array([0, 1, 0, 1], np.int32)
    vals = np.array([c["A11"], c["A12"], c["A21"], c["A22"]], np.float64)
    return rowptr, colind, vals


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "bilu_2x2_worked.json")))["cases"],
                         ids=lambda c: c["name"])
def test_bilu0_worked_example(case):
    rowptr, colind, vals = _case(case)
    X, Dinv, ns = oracle.bilu0_seq(rowptr, colind, vals)
    np.testing.assert_allclose(X[0], case["U11"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(X[1], case["U12"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(X[2], case["L21"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(X[3], case["U22"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(Dinv[0], case["Dinv1"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(Dinv[1], case["Dinv2"], rtol=0, atol=1e-15)
    assert ns == case["singular"]


@pytest.mark.parametrize("maker", [
    lambda: _sys(4, 3, order="natural"),
    lambda: _sys(5, 4, seed=1, order="rcm"),
    lambda: _sys(3, 6, seed=2, order="line"),
    lambda: gen.random_pattern_system(20, 30, seed=3),
    lambda: gen.random_pattern_system(16, 60, seed=4, cfl=1.0),
], ids=["grid_natural", "grid_rcm", "grid_line", "random_triangles", "random_dense_ish"])
def test_bilu0_matches_dense_ikj(maker):
    s = maker()
    X, Dinv, ns = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    L, U = dense.bilu0_ikj(s.rowptr, s.colind, s.vals)
    Xd = dense.pattern_layout_from_dense(s.rowptr, s.colind, L, U)
    assert ns == 0
    assert _rel(X, Xd) < 1e-13
    n = s.n
    Dd = np.array([np.linalg.inv(U[i, i]) for i in range(n)])
    assert _rel(Dinv, Dd) < 1e-12


@pytest.mark.parametrize("maker", [
    lambda: _sys(6, 5, seed=5),
    lambda: gen.random_pattern_system(24, 50, seed=6),
], ids=["grid", "random_triangles"])
def test_bilu0_defining_equations_dense(maker):
    """(LU)_ij = A_ij for every (i,j) in S_B (Eq. bilu), via dense products."""
    s = maker()
    X, Dinv, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    L, U = dense.factors_from_pattern_layout(s.rowptr, s.colind, X)
    LU = dense.blocks_to_dense(L) @ dense.blocks_to_dense(U)
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    mask = np.kron(dense.block_mask(s.rowptr, s.colind), np.ones((4, 4), bool))
    assert np.abs(LU - A)[mask].max() / np.abs(A).max() < 1e-12
    # and the oracle's own defect measure agrees with the dense one
    assert oracle.lu_defect_max(s.rowptr, s.colind, s.vals, X) / np.abs(A).max() < 1e-12


def test_bilu0_defining_equations_sparse_64x64():
    """Same identity on the 64x64 grid workload through scipy sparse products."""
    s = gen.workload("inviscid_64x64")
    X, Dinv, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    n = s.n
    rows = np.repeat(np.arange(n), np.diff(s.rowptr))
    lo = rows > s.colind
    Lv = np.where(lo[:, None, None], X, 0.0)
    Lv[~lo] = 0.0
    Lv[rows == s.colind] = np.eye(4)
    Uv = np.where(lo[:, None, None], 0.0, X)
    Lm = _bsr(s.rowptr, s.colind, Lv).tocsr()
    Um = _bsr(s.rowptr, s.colind, Uv).tocsr()
    LU = (Lm @ Um).tocsr()
    A = _bsr(s.rowptr, s.colind, s.vals).tocsr()
    Am = A.copy()
    Am.data[:] = 1.0
    d = (LU - A).multiply(Am)
    assert np.abs(d.data).max() / np.abs(A.data).max() < 1e-12


def test_full_pattern_is_exact_block_lu():
    """With every block present ILU(0) is the exact block LU: L U = A
    everywhere and the exact apply equals numpy.linalg.solve."""
    s = gen.random_pattern_system(6, 0, seed=8, structure="full")
    X, Dinv, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    L, U = dense.factors_from_pattern_layout(s.rowptr, s.colind, X)
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    assert _rel(dense.blocks_to_dense(L) @ dense.blocks_to_dense(U), A) < 1e-13
    z = oracle.apply(s.rowptr, s.colind, X, Dinv, s.b, -1, -1)
    ref = np.linalg.solve(A, s.b.reshape(-1)).reshape(-1, 4)
    assert _rel(z, ref) < 1e-12


def test_triangle_free_grid_structure():
    """The triangulated quad grid has no 3-cycles, so every off-diagonal pair
    list is empty: at the fixed point U_ij = A_ij (i<j) and L_ij = A_ij U_jj^-1."""
    s = gen.workload("inviscid_64x64")
    n = s.n
    # no 3-cycles: for every edge (i,j) the neighbour sets of i and j are disjoint
    nbrs = [set(s.colind[s.rowptr[i]:s.rowptr[i + 1]]) - {i} for i in range(n)]
    assert all(not (nbrs[i] & nbrs[j]) for i in range(n) for j in nbrs[i])
    assert max(len(x) for x in nbrs) <= 3
    X, Dinv, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    rows = np.repeat(np.arange(n), np.diff(s.rowptr))
    up = rows < s.colind
    np.testing.assert_array_equal(X[up], s.vals[up])
    lo = rows > s.colind
    ref = np.einsum("bij,bjk->bik", s.vals[lo], Dinv[s.colind[lo]])
    assert _rel(X[lo], ref) < 1e-14


# ------------------------------------------------------------ synchronous sweeps

def test_sync_sweeps_reach_sequential_fixed_point_bitwise():
    """Sync sweeps stop changing after finitely many iterations (Theorem on
    the modified Jacobi-type iteration: at most m/b^2 = nnzb), and the point
    they stop at is sequential BILU(0) (uniqueness theorem), bit for bit."""
    s = _sys(8, 6, seed=9)
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    X, D, _ = oracle.bilu_init(s.rowptr, s.colind, s.vals)
    for k in range(1, s.nnzb + 1):
        Xn, Dn, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, X, D)
        if np.array_equal(Xn, X) and np.array_equal(Dn, D):
            break
        X, D = Xn, Dn
    assert k <= s.nnzb
    np.testing.assert_array_equal(X, Xs)
    np.testing.assert_array_equal(D, Ds)
    # each link of a decreasing-neighbour chain costs at most two sweeps
    assert k - 1 <= 2 * _chain_depth(s.rowptr, s.colind) + 2


def test_sync_sweeps_general_pattern_reach_fixed_point():
    s = gen.random_pattern_system(20, 40, seed=10)
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, s.nnzb)
    assert _rel(X, Xs) < 1e-12


def test_sync_sweep_error_decreases_on_64x64():
    s = gen.workload("inviscid_64x64")
    Xs, _, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    X, D, _ = oracle.bilu_init(s.rowptr, s.colind, s.vals)
    errs = []
    for k in range(40):
        X, D, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, X, D)
        errs.append(np.abs(X - Xs).max())
    errs = np.array(errs)
    # each dependency link takes two sweeps (U_kk -> L_ik -> U_ii), so the error
    # decreases over every pair of sweeps, not necessarily every single one
    assert np.all(errs[5::2] <= errs[3:-2:2]) and np.all(errs[6::2] <= errs[4:-2:2])
    assert errs[3] < 0.1 and errs[21] < 1e-10 and errs[39] == 0.0


@pytest.mark.parametrize("structure", ["diagonal", "lower", "upper"])
def test_one_sync_sweep_is_exact_for_block_triangular(structure):
    """From X^0 = A one sweep is exact when A is block diagonal or block
    triangular: no product pair reaches a block whose value changes."""
    s = gen.random_pattern_system(12, 20, seed=11, structure=structure)
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    X1, D1, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    assert _rel(X1, Xs) < 1e-14 and _rel(D1, Ds) < 1e-14
    L, U = dense.bilu0_ikj(s.rowptr, s.colind, s.vals)
    assert _rel(X1, dense.pattern_layout_from_dense(s.rowptr, s.colind, L, U)) < 1e-13
    if structure in ("diagonal", "upper"):
        np.testing.assert_array_equal(X1, s.vals)  # U = A, no L blocks


# ------------------------------------------------- asynchronous (chunked) emulation

def test_one_chunk_one_sweep_is_sequential():
    """One thread, one chunk, one sweep of the in-place iteration is the
    traditional ILU(0) (Sec. 3.3; Sec. 6 setup)."""
    s = gen.workload("inviscid_64x64")
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    X, D, _ = oracle.bilu_init(s.rowptr, s.colind, s.vals)
    oracle.bilu_chunked_sweep(s.rowptr, s.colind, s.vals, X, D, s.n, [0])
    np.testing.assert_array_equal(X, Xs)
    np.testing.assert_array_equal(D, Ds)


@pytest.mark.parametrize("nchunks", [3, 8])
def test_chunked_sweeps_exact_within_chunk_count(nchunks):
    """In-place sweeps over c chunks in any order per sweep are exact after at
    most c sweeps (Sec. 4.2, remark on OpenMP chunks)."""
    s = _sys(6, 6, seed=12)
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    X, D, _ = oracle.bilu_init(s.rowptr, s.colind, s.vals)
    chunk = -(-s.n // nchunks)
    rng = np.random.default_rng(13)
    for _ in range(nchunks):
        oracle.bilu_chunked_sweep(s.rowptr, s.colind, s.vals, X, D, chunk,
                                  rng.permutation(nchunks))
    np.testing.assert_array_equal(X, Xs)
    np.testing.assert_array_equal(D, Ds)


# ------------------------------------------------------------ triangular apply

def test_first_lower_sweep_from_zero_is_rhs():
    s = _sys(5, 5, seed=14)
    X, D, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    y = oracle.lower_sweep(s.rowptr, s.colind, X, s.b, np.zeros_like(s.b))
    np.testing.assert_array_equal(y, s.b)


def test_sweeps_reach_exact_substitution():
    """Jacobi sweeps on a block triangular system are exact after at most n/b
    iterations (Theorem, Sec. 4.1); concretely after depth+1 sweeps."""
    s = _sys(6, 5, seed=15)
    X, D, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    dl = _chain_depth(s.rowptr, s.colind, lower=True)
    du = _chain_depth(s.rowptr, s.colind, lower=False)
    y_exact = oracle.lower_solve(s.rowptr, s.colind, X, s.b)
    z_exact = oracle.upper_solve(s.rowptr, s.colind, X, D, y_exact)
    z = oracle.apply(s.rowptr, s.colind, X, D, s.b, dl + 1, du + 1)
    np.testing.assert_array_equal(z, z_exact)
    z_n = oracle.apply(s.rowptr, s.colind, X, D, s.b, s.n, s.n)
    np.testing.assert_array_equal(z_n, z_exact)
    # one sweep short is generally not exact
    z_short = oracle.apply(s.rowptr, s.colind, X, D, s.b, dl, du + 1)
    assert not np.array_equal(z_short, z_exact)


def test_exact_apply_matches_dense_solve():
    for s in (_sys(5, 4, seed=16), gen.random_pattern_system(18, 30, seed=17)):
        X, D, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
        L, U = dense.factors_from_pattern_layout(s.rowptr, s.colind, X)
        z = oracle.apply(s.rowptr, s.colind, X, D, s.b, -1, -1)
        assert _rel(z, dense.lu_solve_dense(L, U, s.b)) < 1e-11


def test_block_diagonal_one_sweep_exact():
    s = gen.random_pattern_system(10, 0, seed=18, structure="diagonal")
    X, D, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    z = oracle.apply(s.rowptr, s.colind, X, D, s.b, 1, 1)
    ref = np.stack([np.linalg.solve(s.vals[i], s.b[i]) for i in range(s.n)])
    assert _rel(z, ref) < 1e-13


def test_jacobi_sweep_matches_dense_iteration():
    """One lower / upper Jacobi sweep equals the dense splitting iteration
    x' = D^{-1}(b - (T - D) x) of the block triangular matrix T (Sec. 4.1)."""
    s = gen.random_pattern_system(14, 25, seed=19)
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 2)
    L, U = dense.factors_from_pattern_layout(s.rowptr, s.colind, X)
    rng = np.random.default_rng(20)
    yin = rng.standard_normal(s.b.shape)
    Ld = dense.blocks_to_dense(L)
    y = oracle.lower_sweep(s.rowptr, s.colind, X, s.b, yin)
    ref = s.b.reshape(-1) - (Ld - np.eye(Ld.shape[0])) @ yin.reshape(-1)
    assert _rel(y.reshape(-1), ref) < 1e-13
    Ublk = U.copy()
    for i in range(s.n):
        Ublk[i, i] = 0
    xin = rng.standard_normal(s.b.shape)
    x = oracle.upper_sweep(s.rowptr, s.colind, X, D, s.b, xin)
    Dinv_d = dense.blocks_to_dense(np.array([[D[i] if i == j else np.zeros((4, 4))
                                              for j in range(s.n)] for i in range(s.n)]))
    ref = Dinv_d @ (s.b.reshape(-1) - dense.blocks_to_dense(Ublk) @ xin.reshape(-1))
    assert _rel(x.reshape(-1), ref) < 1e-12


# ------------------------------------------------------------------------ SpMV

def test_spmv_matches_scipy_and_dense():
    s = gen.workload("inviscid_64x64")
    x = np.random.default_rng(21).standard_normal(s.b.shape)
    y = oracle.spmv(s.rowptr, s.colind, s.vals, x)
    ref = _bsr(s.rowptr, s.colind, s.vals) @ x.reshape(-1)
    assert _rel(y.reshape(-1), ref) < 1e-15
    t = _sys(4, 3, seed=22)
    xt = np.random.default_rng(23).standard_normal(t.b.shape)
    yt = oracle.spmv(t.rowptr, t.colind, t.vals, xt)
    assert _rel(yt.reshape(-1), dense.to_dense(t.rowptr, t.colind, t.vals) @ xt.reshape(-1)) < 1e-15


# ---------------------------------------------------------------------- FGMRES

def _krylov_min_residual(Bop, b, k):
    """min_y ||b - B K y|| over the k-dim Krylov space K of B and b (dense)."""
    K = np.zeros((len(b), k))
    v = b / np.linalg.norm(b)
    for j in range(k):
        K[:, j] = v
        v = Bop @ v
        for i in range(j + 1):  # orthogonalise twice for a clean basis
            v -= K[:, i] * (K[:, i] @ v)
        for i in range(j + 1):
            v -= K[:, i] * (K[:, i] @ v)
        v /= np.linalg.norm(v)
    y, *_ = np.linalg.lstsq(Bop @ K, b, rcond=None)
    return np.linalg.norm(b - Bop @ K @ y)


def test_fgmres_residual_is_krylov_minimum():
    """With a fixed (linear) preconditioner M^-1, FGMRES's residual estimate
    after k steps is min ||b - A M^-1 v|| over the Krylov space of A M^-1."""
    s = _sys(4, 3, seed=24, cfl=1.0)
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    nv = s.n * 4
    Minv = np.zeros((nv, nv))
    for c in range(nv):
        e = np.zeros(nv)
        e[c] = 1.0
        Minv[:, c] = oracle.apply(s.rowptr, s.colind, X, D, e.reshape(-1, 4), 2, 2).reshape(-1)
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    Bop = A @ Minv
    b = s.b.reshape(-1)
    _, res = oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, s.b, 2, 2, restart=nv,
                           max_iters=12, rtol=1e-14)
    for k in range(1, 9):
        ref = _krylov_min_residual(Bop, b, k) / np.linalg.norm(b)
        assert abs(res.history[k] - ref) <= 1e-9 * max(ref, 1e-300) + 1e-13


def test_fgmres_solution_matches_numpy_solve():
    s = _sys(4, 3, seed=25)
    X, D, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    x, res = oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, s.b, -1, -1, restart=48,
                           max_iters=200, rtol=1e-10)
    assert res.converged and res.rel_resid_true <= 1e-10
    ref = np.linalg.solve(dense.to_dense(s.rowptr, s.colind, s.vals), s.b.reshape(-1))
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    bound = np.linalg.cond(A) * 1e-10 * 10
    assert _rel(x.reshape(-1), ref) < bound


@pytest.mark.parametrize("structure", ["diagonal", "full"])
def test_fgmres_exact_preconditioner_one_iteration(structure):
    """When block ILU(0) is exact (block diagonal or full pattern) M = A and
    FGMRES converges in one step."""
    s = gen.random_pattern_system(8, 0, seed=26, structure=structure)
    X, D, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    x, res = oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, s.b, -1, -1, restart=30,
                           rtol=1e-8)
    assert res.iters == 1 and res.converged


def test_fgmres_64x64_workload_settings():
    """The 64x64 workload with 4 sync build sweeps and 3+3 apply sweeps:
    converges, true residual <= rtol, estimate monotone within each cycle."""
    s = gen.workload("inviscid_64x64")
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 4)
    x, res = oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, s.b, 3, 3, restart=30, rtol=1e-6)
    assert res.converged and res.rel_resid_true <= 1e-6
    h = res.history
    assert np.all(np.diff(h[: min(len(h), 31)]) <= 1e-15)
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x)
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6


def test_fgmres_restarts_and_monotone_cycles():
    s = _sys(6, 6, seed=27, cfl=1.0)
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    x, res = oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, s.b, 1, 1, restart=4,
                           max_iters=400, rtol=1e-8)
    assert res.converged and res.restarts >= 2
    h = res.history
    for c in range(res.restarts):
        seg = h[1 + 4 * c: 1 + 4 * (c + 1)]
        assert np.all(np.diff(seg) <= 1e-15)


def test_fgmres_zero_rhs():
    s = _sys(3, 3, seed=28)
    X, D, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    x, res = oracle.fgmres(s.rowptr, s.colind, s.vals, X, D, np.zeros_like(s.b), 3, 3)
    assert res.converged and res.iters == 0 and not np.any(x)


# ----------------------------------------------------------------- diagnostics

def test_ilu_residual_zero_at_fixed_point_and_closed_form():
    s = _sys(6, 4, seed=29)
    Xs, _, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    assert oracle.ilu_residual_l1(s.rowptr, s.colind, s.vals, Xs) == 0.0
    # block lower triangular A: h(X^0) changes only L: L_ij = A_ij A_jj^-1
    t = gen.random_pattern_system(10, 15, seed=30, structure="lower")
    X0, _, _ = oracle.bilu_init(t.rowptr, t.colind, t.vals)
    rows = np.repeat(np.arange(t.n), np.diff(t.rowptr))
    lo = rows > t.colind
    dpos = t.rowptr[1:] - 1  # diagonal is last in each row of a lower pattern
    ref = np.abs(t.vals[lo] - np.einsum("bij,bjk->bik", t.vals[lo],
                                       np.linalg.inv(t.vals[dpos[t.colind[lo]]]))).sum()
    got = oracle.ilu_residual_l1(t.rowptr, t.colind, t.vals, X0)
    assert abs(got - ref) <= 1e-12 * ref


def test_jacobi_norms_match_dense():
    s = gen.random_pattern_system(12, 20, seed=31)
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 3)
    ln, un = oracle.jacobi_norms(s.rowptr, s.colind, X, D)
    L, U = dense.factors_from_pattern_layout(s.rowptr, s.colind, X)
    Ld = dense.blocks_to_dense(L) - np.eye(4 * s.n)
    assert abs(ln - np.abs(Ld).sum(axis=1).max()) < 1e-12 * ln
    Uoff = U.copy()
    for i in range(s.n):
        Uoff[i, i] = 0
    Dd = dense.blocks_to_dense(np.array([[D[i] if i == j else np.zeros((4, 4))
                                          for j in range(s.n)] for i in range(s.n)]))
    un_ref = np.abs(Dd @ dense.blocks_to_dense(Uoff)).sum(axis=1).max()
    assert abs(un - un_ref) < 1e-12 * un_ref
    d = gen.random_pattern_system(6, 0, seed=32, structure="diagonal")
    Xd, Dd2, _ = oracle.bilu0_seq(d.rowptr, d.colind, d.vals)
    assert oracle.jacobi_norms(d.rowptr, d.colind, Xd, Dd2) == (0.0, 0.0)


def test_singular_pivot_counted_in_sweeps():
    """A zero diagonal block is replaced (modified iteration, Sec. 4.2)."""
    s = _sys(3, 3, seed=33)
    A = s.vals.copy()
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    d0 = np.flatnonzero((rows == 0) & (s.colind == 0))[0]
    A[d0] = 0.0
    X, D, ns = oracle.bilu_init(s.rowptr, s.colind, A)
    assert ns == 1
    np.testing.assert_array_equal(D[0], np.eye(4))
    X, D, ns = oracle.bilu_sync_sweep(s.rowptr, s.colind, A, X, D)
    assert ns == 1
