"""Pins of the CPU oracle's scalar ILU(0) (Chow-Patel, the variant the paper
compares against, Sec. 3.2) against facts fixed by mathematics: the textbook
masked IKJ elimination in numpy (oracle/dense.py, written independently), the
defining equations (LU)_ij = A_ij on the scalar pattern, exact LU on a full
pattern, closed forms for triangular matrices, and numpy solves."""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle
from oracle import dense


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


MAKERS = {
    "grid_natural": lambda: gen.small_system(4, 3, seed=0, order="natural"),
    "grid_rcm": lambda: gen.small_system(5, 4, seed=1),
    "random_triangles": lambda: gen.random_pattern_system(14, 25, seed=3),
    "random_weak": lambda: gen.random_pattern_system(12, 40, seed=4, cfl=1.0),
}


@pytest.mark.parametrize("name", list(MAKERS))
def test_silu0_matches_dense_ikj(name):
    s = MAKERS[name]()
    X, ns = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    assert ns == 0
    L, U = dense.silu0_ikj(s.rowptr, s.colind, s.vals)
    Lo, Uo = dense.scalar_factors_dense(s.rowptr, s.colind, X)
    mask = dense.scalar_mask(s.rowptr, s.colind)
    assert _rel(np.where(mask, Lo, 0), np.where(mask, L, 0)) < 1e-13
    assert _rel(np.where(mask, Uo, 0), np.where(mask, U, 0)) < 1e-13


@pytest.mark.parametrize("name", ["grid_rcm", "random_triangles"])
def test_silu0_defining_equations(name):
    """(L U)_ij = A_ij for every (i, j) of the scalar pattern."""
    s = MAKERS[name]()
    X, _ = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    L, U = dense.scalar_factors_dense(s.rowptr, s.colind, X)
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    mask = dense.scalar_mask(s.rowptr, s.colind)
    assert np.abs(np.where(mask, L @ U - A, 0.0)).max() < 1e-12 * np.abs(A).max()


def test_full_pattern_is_exact_lu():
    s = gen.random_pattern_system(6, 0, seed=5, structure="full")
    X, ns = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    L, U = dense.scalar_factors_dense(s.rowptr, s.colind, X)
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    assert ns == 0 and _rel(L @ U, A) < 1e-13
    z = oracle.silu_apply(s.rowptr, s.colind, X, s.b, -1, -1)
    assert _rel(z.reshape(-1), np.linalg.solve(A, s.b.reshape(-1))) < 1e-12


def test_sync_sweeps_reach_sequential_bitwise():
    """The Jacobi-type iteration of Eq. (scalarilu_fp) from X^0 = A stops
    changing at the sequential ILU(0) (its unique fixed point)."""
    s = gen.small_system(4, 3, seed=7)
    Xs, _ = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    X = s.vals.copy()
    for k in range(400):
        Xn, _ = oracle.silu_sync(s.rowptr, s.colind, s.vals, 1, X0=X)
        if np.array_equal(Xn, X):
            break
        X = Xn
    assert np.array_equal(X, Xs), k


@pytest.mark.parametrize("structure", ["diagonal", "lower", "upper"])
def test_one_sync_sweep_is_exact_for_triangular(structure):
    """Diagonal blocks here are diagonal matrices, so block-triangular A is
    scalar triangular: from X^0 = A one sweep gives L_ij = A_ij / A_jj (lower)
    or U = A (upper, diagonal)."""
    s = gen.random_pattern_system(10, 20, seed=11, structure=structure)
    Xs, _ = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    X1, _ = oracle.silu_sync(s.rowptr, s.colind, s.vals, 1)
    assert _rel(X1, Xs) < 1e-15
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    L, U = dense.scalar_factors_dense(s.rowptr, s.colind, X1)
    if structure == "lower":
        d = np.diag(A)
        assert _rel(np.tril(L, -1), np.tril(A, -1) / d[None, :]) < 1e-15
    else:
        np.testing.assert_array_equal(X1, s.vals)


def test_triangular_sweeps():
    s = MAKERS["random_triangles"]()
    X, _ = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    L, U = dense.scalar_factors_dense(s.rowptr, s.colind, X)
    r = np.random.default_rng(2).standard_normal((s.n, 4))
    # first lower sweep from zero gives the right-hand side
    y1 = oracle.silu_lower_sweep(s.rowptr, s.colind, X, r, np.zeros_like(r))
    np.testing.assert_array_equal(y1, r)
    # a sweep is the dense Jacobi iteration y <- r - (L - I) y, x <- D^-1 (y - (U - D) x)
    y0 = np.random.default_rng(3).standard_normal((s.n, 4))
    y = oracle.silu_lower_sweep(s.rowptr, s.colind, X, r, y0)
    assert _rel(y.reshape(-1), r.reshape(-1) - (L - np.eye(4 * s.n)) @ y0.reshape(-1)) < 1e-13
    D = np.diag(np.diag(U))
    x = oracle.silu_upper_sweep(s.rowptr, s.colind, X, r, y0)
    ref = np.linalg.solve(D, r.reshape(-1) - (U - D) @ y0.reshape(-1))
    assert _rel(x.reshape(-1), ref) < 1e-13
    # exact substitution = dense solve with the factors; enough sweeps reach it
    z = oracle.silu_apply(s.rowptr, s.colind, X, r, -1, -1)
    zd = np.linalg.solve(U, np.linalg.solve(L, r.reshape(-1)))
    assert _rel(z.reshape(-1), zd) < 1e-12
    zs = oracle.silu_apply(s.rowptr, s.colind, X, r, 4 * s.n, 4 * s.n)
    assert _rel(zs, z) < 1e-12


@pytest.mark.parametrize("structure", ["diagonal", "full"])
def test_fgmres_exact_scalar_preconditioner_one_iteration(structure):
    s = gen.random_pattern_system(6, 0, seed=26, structure=structure)
    X, _ = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    x, res = oracle.fgmres(s.rowptr, s.colind, s.vals, X, None, s.b, -1, -1, restart=30,
                           rtol=1e-8)
    assert res.iters == 1 and res.converged


def test_zero_pivot_replaced_and_counted():
    """U_00 = A_00 has no update before it: zeroing it makes every L entry of
    column 0 divide by a zero pivot, which the modified iteration replaces by 1
    (so those entries equal their residual)."""
    s = gen.small_system(3, 3, seed=8)
    vals = s.vals.copy()
    vals[s.rowptr[0], 0, 0] = 0.0          # block (0,0) is first in row 0
    X, ns = oracle.silu0_seq(s.rowptr, s.colind, vals)
    assert ns >= 1 and np.all(np.isfinite(X))
    L, U = dense.scalar_factors_dense(s.rowptr, s.colind, X)
    A = dense.to_dense(s.rowptr, s.colind, vals)
    mask = dense.scalar_mask(s.rowptr, s.colind)
    col0 = np.flatnonzero(mask[:, 0])[1:]  # L entries of column 0: A_i0 / 1
    np.testing.assert_array_equal(L[col0, 0], A[col0, 0])
