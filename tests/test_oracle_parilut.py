"""Pins of the oracle's threshold block ILU (fill of L U added, largest blocks
kept, synchronous sweeps in between).

The paper names a parallel threshold ILU as the next extension of its sweeps
without giving one, so the oracle states the library's loop and these tests
pin its parts to independent facts: the pattern of L U against a boolean
matrix product, the selection against the properties that define it, and the
whole loop with unlimited fill against the exact block LU of dense numpy
elimination.
"""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle
from oracle import dense

SYSTEMS = {
    "grid6x5": lambda: gen.small_system(6, 5, seed=1),
    "random_triangles": lambda: gen.random_pattern_system(40, 60, seed=4),
    "aniso10x6": lambda: gen.small_system(10, 6, seed=3, cfl=1e4, wall_normal_scale=100.0),
}


def _mask(rowptr, colind):
    return dense.block_mask(rowptr, colind)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_lu_pattern_is_the_boolean_product(name):
    s = SYSTEMS[name]()
    M = _mask(s.rowptr, s.colind)
    Lm = (np.tril(M, -1) | np.eye(s.n, dtype=bool)).astype(int)
    Um = np.triu(M).astype(int)
    rp, ci = oracle.lu_pattern(s.rowptr, s.colind)
    assert np.array_equal(_mask(rp, ci), (Lm @ Um) > 0)
    assert all(np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0) for i in range(s.n))
    assert np.all(_mask(rp, ci) >= M)   # the pattern of L U contains the pattern


def test_keep_largest_properties():
    """At most `budget` kept; every kept key above every dropped one; the
    largest dropped group (equal keys) would not fit: these fix the set."""
    rng = np.random.default_rng(5)
    for trial in range(50):
        m = int(rng.integers(1, 60))
        key = rng.integers(0, 12, size=m).astype(float)   # many ties
        budget = int(rng.integers(0, m + 3))
        keep = oracle.keep_largest(key, budget)
        assert keep.sum() <= budget
        if keep.any() and (~keep).any():
            assert key[keep].min() > key[~keep].max()
        if (~keep).any():
            top_dropped = key[~keep].max()
            assert keep.sum() + np.sum(key == top_dropped) > budget
    assert oracle.keep_largest(np.array([3.0, 1, 2, 2, 5]), 3).tolist() == [True, False, False, False, True]


def test_no_iterations_is_block_ilu_sweeps():
    s = SYSTEMS["grid6x5"]()
    rp, ci, X, D = oracle.parilut(s.rowptr, s.colind, s.vals, fill=2.0, iters=0, sweeps=3)
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 3)
    assert np.array_equal(rp, s.rowptr) and np.array_equal(ci, s.colind)
    assert np.array_equal(X, Xo) and np.array_equal(D, Do)


def test_unlimited_fill_reaches_the_exact_block_lu():
    """With no dropping the pattern closes under fill: it becomes the block
    structure of the exact LU factors, and the sweeps reach them: L U = A
    (numpy dense elimination with no pattern restriction gives the factors)."""
    s = gen.random_pattern_system(12, 6, seed=8)
    rp, ci, X, D = oracle.parilut(s.rowptr, s.colind, s.vals, fill=1e6, iters=12, sweeps=3)
    full_rp = np.arange(0, s.n * s.n + 1, s.n, dtype=np.int32)
    full_ci = np.tile(np.arange(s.n, dtype=np.int32), s.n)
    full_vals = dense.to_blocks(s.rowptr, s.colind, s.vals).reshape(-1, 4, 4)
    L, U = dense.bilu0_ikj(full_rp, full_ci, full_vals)   # full pattern: the exact block LU
    nz = (np.abs(L).sum(axis=(2, 3)) + np.abs(U).sum(axis=(2, 3))) > 0
    assert np.array_equal(_mask(rp, ci), nz)
    Lx, Ux = dense.factors_from_pattern_layout(rp, ci, X)
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    LU = dense.blocks_to_dense(Lx) @ dense.blocks_to_dense(Ux)
    assert np.abs(LU - A).max() / np.abs(A).max() < 1e-12


@pytest.mark.parametrize("fill", [1.0, 1.5, 2.0])
def test_budgets_and_diagonal(fill):
    s = SYSTEMS["aniso10x6"]()
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    bl = int(np.floor(fill * np.sum(rows > s.colind)))
    bu = int(np.floor(fill * np.sum(rows < s.colind)))
    rp, ci, X, D = oracle.parilut(s.rowptr, s.colind, s.vals, fill=fill, iters=3, sweeps=2)
    r = np.repeat(np.arange(s.n), np.diff(rp))
    assert np.sum(r > ci) <= bl and np.sum(r < ci) <= bu
    assert np.array_equal(np.sort(ci[r == ci]), np.arange(s.n))


def test_threshold_ilu_cuts_iterations():
    """More (selected) fill, a better preconditioner: fewer FGMRES iterations
    than block ILU(0) with the same sweep counts on the anisotropic grid."""
    s = gen.small_system(40, 20, seed=3, cfl=1e4, wall_normal_scale=100.0)
    X0, D0, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 8)
    _, r0 = oracle.fgmres(s.rowptr, s.colind, s.vals, X0, D0, s.b, 6, 6, restart=50)
    rp, ci, X, D = oracle.parilut(s.rowptr, s.colind, s.vals, fill=2.0, iters=3, sweeps=2)
    x, r1 = oracle.fgmres_ilu_pattern(s.rowptr, s.colind, s.vals, rp, ci, X, D, s.b, 6, 6,
                                      restart=50)
    assert r1.converged and r1.iters < r0.iters
    res = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x)
    assert np.linalg.norm(res) / np.linalg.norm(s.b) <= 1e-6


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_fix_constant_upper(name):
    """Exactly the strictly upper blocks with no product pair (no k < i with
    (i,k) and (k,j) in the pattern: the strict-lower by strict-upper boolean
    product is zero there) take A's value; on the triangle-free grids that is
    every strictly upper block."""
    s = SYSTEMS[name]()
    rng = np.random.default_rng(3)
    X = rng.standard_normal(s.vals.shape)
    Y = oracle.fix_constant_upper(s.rowptr, s.colind, s.vals, X)
    M = _mask(s.rowptr, s.colind).astype(int)
    has_pair = (np.tril(M, -1) @ np.triu(M, 1)) > 0
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    const = (rows < s.colind) & ~has_pair[rows, s.colind]
    assert np.array_equal(Y[const], s.vals[const]) and np.array_equal(Y[~const], X[~const])
    if name != "random_triangles":
        assert np.array_equal(const, rows < s.colind)
