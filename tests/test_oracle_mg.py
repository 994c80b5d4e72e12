"""Pins of the oracle's multigrid cycle with block ILU smoothing.

The paper names block ILU iterations as fine-grain parallel multigrid
smoothers (and the study of their smoothing property) as future work without
fixing a cycle, so the oracle states the library's cycle plainly and these
tests pin it to things other than itself: hand-worked aggregations
(tests/golden), structural invariants, numpy dense products P^T A P, the
ILU-preconditioned Richardson iteration written with numpy.linalg.solve, and the
two- and three-level error-propagation operators of the cycle built from dense
matrices.
"""
import json
import os

import numpy as np
import pytest

import abilu_inputs as gen
import oracle
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _graph_system(n, edges):
    """BSR arrays with s*I off-diagonal blocks (both directions) and 10*I diagonals."""
    ent = {(i, i): 10.0 for i in range(n)}
    for u, v, s in edges:
        ent[(int(u), int(v))] = float(s)
        ent[(int(v), int(u))] = float(s)
    keys = sorted(ent)
    rowptr = np.zeros(n + 1, np.int32)
    for i, _ in keys:
        rowptr[i + 1] += 1
    rowptr = np.cumsum(rowptr).astype(np.int32)
    colind = np.array([j for _, j in keys], np.int32)
    vals = np.array([ent[k] * np.eye(4) for k in keys])
    return rowptr, colind, vals


def _P(agg, nc):
    """Dense piecewise-constant prolongation (4n x 4nc)."""
    n = len(agg)
    P = np.zeros((4 * n, 4 * nc))
    for i, a in enumerate(agg):
        P[4 * i:4 * i + 4, 4 * a:4 * a + 4] = np.eye(4)
    return P


GRIDS = {
    "grid6x5": lambda: gen.small_system(6, 5, seed=1),
    "grid12x9_natural": lambda: gen.small_system(12, 9, seed=2, order="natural"),
    "random_triangles": lambda: gen.random_pattern_system(60, 150, seed=4),
    "aniso10x6": lambda: gen.small_system(10, 6, seed=3, cfl=1e4, wall_normal_scale=100.0,
                                          order="natural"),
}


# ------------------------------------------------------------- aggregation

def test_aggregation_hand_worked():
    d = json.load(open(os.path.join(GOLDEN, "mg_aggregation_worked.json")))
    for case in d["cases"]:
        rp, ci, vals = _graph_system(case["n"], case["edges"])
        agg, nc = oracle.mg_aggregate(rp, ci, vals, d["theta"])
        assert nc == case["nc"], case["name"]
        assert agg.tolist() == case["agg"], case["name"]


def test_aggregation_block_diagonal_gives_singletons():
    s = gen.random_pattern_system(20, 0, seed=9, structure="diagonal")
    agg, nc = oracle.mg_aggregate(s.rowptr, s.colind, s.vals, 0.25)
    assert nc == s.n and sorted(agg.tolist()) == list(range(s.n))


@pytest.mark.parametrize("name", list(GRIDS))
def test_aggregation_invariants(name):
    """A partition of the cells into connected aggregates, numbered densely;
    each pass-1 aggregate holds its root's strong neighbours."""
    s = GRIDS[name]()
    theta = 0.25
    agg, nc = oracle.mg_aggregate(s.rowptr, s.colind, s.vals, theta)
    assert agg.min() == 0 and agg.max() == nc - 1
    assert np.all(np.bincount(agg, minlength=nc) > 0)
    nbr = [s.colind[s.rowptr[i]:s.rowptr[i + 1]] for i in range(s.n)]
    for a in range(nc):
        cells = set(np.flatnonzero(agg == a).tolist())
        seen, todo = set(), [min(cells)]
        while todo:
            c = todo.pop()
            if c in seen:
                continue
            seen.add(c)
            todo += [int(j) for j in nbr[c] if int(j) in cells]
        assert seen == cells, (name, a)
    # the first cell of aggregate 0 is cell 0's root (cell 0 has strong neighbours
    # in these systems): it roots aggregate 0 with all its strong neighbours
    norms = np.array([np.sum(b * b) for b in s.vals])
    row0 = range(s.rowptr[0], s.rowptr[1])
    off = [p for p in row0 if s.colind[p] != 0]
    mx = max(norms[p] for p in off)
    strong = [int(s.colind[p]) for p in off if norms[p] >= theta * theta * mx]
    assert agg[0] == 0 and all(agg[j] == 0 for j in strong)


def test_aggregation_follows_strong_direction():
    """Wall-normal couplings 100x stronger: every aggregate lies inside one
    wall-normal column of the natural numbering (cell 2q + t, quad q = j nx + i)."""
    nx, ny = 10, 6
    s = gen.small_system(nx, ny, seed=3, cfl=1e4, wall_normal_scale=100.0, order="natural")
    agg, nc = oracle.mg_aggregate(s.rowptr, s.colind, s.vals, 0.25)
    col = (np.arange(s.n) // 2) % nx
    for a in range(nc):
        assert len(set(col[agg == a].tolist())) == 1, a
    assert nc < s.n / 2.5   # still coarsens (about 3 cells per aggregate or more)


# ---------------------------------------------------------------- Galerkin

@pytest.mark.parametrize("name", list(GRIDS))
def test_galerkin_equals_dense_product(name):
    s = GRIDS[name]()
    agg, nc = oracle.mg_aggregate(s.rowptr, s.colind, s.vals, 0.25)
    rpc, cic, Ac = oracle.galerkin(s.rowptr, s.colind, s.vals, agg, nc)
    P = _P(agg, nc)
    ref = P.T @ dense.to_dense(s.rowptr, s.colind, s.vals) @ P
    assert _rel(dense.to_dense(rpc, cic, Ac), ref) < 1e-14
    # pattern: block (I, J) present exactly when some block of A maps to it
    M = dense.block_mask(s.rowptr, s.colind).astype(int)
    Pb = np.zeros((s.n, nc), int)
    Pb[np.arange(s.n), agg] = 1
    assert np.array_equal(dense.block_mask(rpc, cic), (Pb.T @ M @ Pb) > 0)
    assert all(np.all(np.diff(cic[rpc[I]:rpc[I + 1]]) > 0) for I in range(nc))


# ---------------------------------------------------------------- V-cycle

def _dense_M(L):
    Ld, Ud = dense.factors_from_pattern_layout(L.rowptr, L.colind, L.X)
    return dense.blocks_to_dense(Ld) @ dense.blocks_to_dense(Ud)


def test_single_level_is_ilu_richardson():
    """One level: the cycle is k steps of x += M^{-1}(b - A x) from 0 with
    M = L U (exact triangular solves), written here with numpy.linalg.solve."""
    s = gen.small_system(6, 5, seed=1)
    lv = oracle.mg_hierarchy(s.rowptr, s.colind, s.vals, max_levels=1, build_sweeps=3)
    assert len(lv) == 1
    A = dense.to_dense(s.rowptr, s.colind, s.vals)
    M = _dense_M(lv[0])
    b = s.b.reshape(-1)
    for k in (1, 2, 5):
        x = np.zeros_like(b)
        for _ in range(k):
            x = x + np.linalg.solve(M, b - A @ x)
        z = oracle.mg_vcycle(lv, s.b, -1, -1, coarse=k)
        assert _rel(z.reshape(-1), x) < 1e-12, k


def _cycle_operator(lv, l, pre, post, coarse_inv):
    """Dense B_l with z = B_l r for the V-cycle from level l, exact smoother
    solves, built from the error propagation operator
        E_l = (I - M^{-1} A)^post (I - P B_{l+1} P^T A) (I - M^{-1} A)^pre,
    B_l = (I - E_l) A^{-1}; on the coarsest level B = coarse_inv(A)."""
    L = lv[l]
    A = dense.to_dense(L.rowptr, L.colind, L.A)
    if l == len(lv) - 1:
        return coarse_inv(A)
    n4 = A.shape[0]
    I = np.eye(n4)
    S = I - np.linalg.solve(_dense_M(L), A)
    P = _P(L.agg, len(lv[l + 1].rowptr) - 1)
    Bc = _cycle_operator(lv, l + 1, pre, post, coarse_inv)
    E = np.linalg.matrix_power(S, post) @ (I - P @ Bc @ P.T @ A) @ np.linalg.matrix_power(S, pre)
    return (I - E) @ np.linalg.inv(A)


@pytest.mark.parametrize("pre,post", [(0, 1), (1, 0), (1, 1), (2, 1)])
def test_two_level_cycle_matches_error_propagation(pre, post):
    """Two levels with the coarse level solved to convergence (many exact-ILU
    Richardson steps): z = (I - E) A^{-1} r with the two-grid operator E."""
    s = gen.small_system(6, 5, seed=1)
    lv = oracle.mg_hierarchy(s.rowptr, s.colind, s.vals, max_levels=2, min_coarse=4,
                             build_sweeps=3)
    assert len(lv) == 2
    z = oracle.mg_vcycle(lv, s.b, -1, -1, pre=pre, post=post, coarse=200)
    B = _cycle_operator(lv, 0, pre, post, np.linalg.inv)
    assert _rel(z.reshape(-1), B @ s.b.reshape(-1)) < 1e-10


def test_three_level_cycle_matches_recursive_operator():
    """Three levels: the middle level's cycle replaces the exact coarse solve of
    the two-grid operator (recursively); coarsest level k Richardson steps."""
    s = gen.small_system(12, 9, seed=2)
    lv = oracle.mg_hierarchy(s.rowptr, s.colind, s.vals, max_levels=3, min_coarse=4,
                             build_sweeps=3)
    assert len(lv) == 3
    k = 3

    def richardson(A):
        # B with z = B r for k steps x += M^{-1}(r - A x) from 0 on the coarsest level
        M = _dense_M(lv[-1])
        S = np.eye(A.shape[0]) - np.linalg.solve(M, A)
        return (np.eye(A.shape[0]) - np.linalg.matrix_power(S, k)) @ np.linalg.inv(A)

    z = oracle.mg_vcycle(lv, s.b, -1, -1, pre=1, post=1, coarse=k)
    B = _cycle_operator(lv, 0, 1, 1, richardson)
    assert _rel(z.reshape(-1), B @ s.b.reshape(-1)) < 1e-10


def test_hierarchy_stopping_rule():
    s = gen.small_system(12, 9, seed=2)
    lv = oracle.mg_hierarchy(s.rowptr, s.colind, s.vals, max_levels=10, min_coarse=20)
    sizes = [len(L.rowptr) - 1 for L in lv]
    assert all(a > b for a, b in zip(sizes, sizes[1:]))
    assert sizes[-1] <= 20 or len(lv) == 10
    assert all(sz > 20 for sz in sizes[:-1])
    assert lv[-1].agg is None and all(L.agg is not None for L in lv[:-1])


# ----------------------------------------------------------------- FGMRES

def test_fgmres_mg_one_level_one_step_is_plain_fgmres():
    """One level and one smoothing step: the cycle is M^{-1} r itself (the
    first step from x = 0), so FGMRES runs the plain block-ILU solve bit for bit."""
    s = gen.workload("inviscid_64x64")
    lv = oracle.mg_hierarchy(s.rowptr, s.colind, s.vals, max_levels=1, build_sweeps=4)
    x1, r1 = oracle.fgmres_mg(lv, s.b, 3, 3, coarse=1)
    x2, r2 = oracle.fgmres(s.rowptr, s.colind, s.vals, lv[0].X, lv[0].Dinv, s.b, 3, 3)
    assert r1.iters == r2.iters and np.array_equal(x1, x2)


def test_fgmres_mg_converges_in_fewer_iterations():
    s = gen.workload("inviscid_64x64")
    lv = oracle.mg_hierarchy(s.rowptr, s.colind, s.vals, min_coarse=64, build_sweeps=4)
    assert len(lv) >= 3
    x, r = oracle.fgmres_mg(lv, s.b, 3, 3, pre=1, post=1, coarse=2)
    assert r.converged and r.rel_resid_true <= 1e-6
    res = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x)
    assert np.linalg.norm(res) / np.linalg.norm(s.b) <= 1e-6
    _, r0 = oracle.fgmres(s.rowptr, s.colind, s.vals, lv[0].X, lv[0].Dinv, s.b, 3, 3)
    assert r.iters < r0.iters
