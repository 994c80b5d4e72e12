"""The FP32 sweep error bound (tests/fp32_bounds.py) pinned on the CPU before
it judges the GPU: an FP32 emulation of one sweep of Eq. (bilu) stays inside
it, and the oracle's sweep with one planted defect (a dropped product pair, a
transposed product, the previous iterate's Dinv) falls outside it."""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle
from fp32_bounds import U32, sweep_bound

f32 = np.float32


def _pairs(rowptr, colind, i, j):
    """(position of L_ik, position of U_kj) for k < min(i, j), ascending k."""
    out = []
    for q in range(rowptr[i], rowptr[i + 1]):
        k = colind[q]
        if k >= min(i, j):
            break
        row = colind[rowptr[k]:rowptr[k + 1]]
        r = int(np.searchsorted(row, j))
        if r < len(row) and row[r] == j:
            out.append((q, rowptr[k] + r))
    return out


def fp32_sweep(s, X, D):
    """One sweep in FP32 arithmetic from FP32-representable X, D: A rounded to
    FP32, each pair's 4x4 product row summed in FP32 and subtracted, L = S Dinv_j
    in FP32, Dinv_i the FP32 rounding of the exact inverse of the FP32 U_ii."""
    n = s.n
    Xo = np.empty_like(X)
    Do = np.empty_like(D)
    X32, D32 = X.astype(f32), D.astype(f32)
    for i in range(n):
        for p in range(s.rowptr[i], s.rowptr[i + 1]):
            j = s.colind[p]
            S = s.vals[p].astype(f32)
            for q, r in _pairs(s.rowptr, s.colind, i, j):
                acc = np.zeros((4, 4), f32)
                for k in range(4):
                    acc = (acc + np.outer(X32[q][:, k], X32[r][k, :])).astype(f32)
                S = (S - acc).astype(f32)
            if j < i:
                o = np.zeros((4, 4), f32)
                for k in range(4):
                    o = (o + np.outer(S[:, k], D32[j][k, :])).astype(f32)
                Xo[p] = o
            else:
                Xo[p] = S
                if j == i:
                    Do[i] = np.linalg.inv(S.astype(np.float64)).astype(f32)
    return Xo, Do


@pytest.fixture(scope="module")
def case():
    s = gen.random_pattern_system(60, 150, seed=4)
    X, D, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 2)
    X, D = X.astype(f32).astype(np.float64), D.astype(f32).astype(np.float64)
    Xo, Do, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, X, D)
    EX, ED = sweep_bound(s, X, D)
    return s, X, D, Xo, Do, EX, ED


def _inside(err, bound, ref):
    return bool((err <= bound + 1e-14 * np.abs(ref).max()).all())


def test_fp32_emulation_is_inside_the_bound(case):
    s, X, D, Xo, Do, EX, ED = case
    Xe, De = fp32_sweep(s, X, D)
    assert _inside(np.abs(Xe - Xo), EX, Xo)
    assert _inside(np.abs(De - Do), ED, Do)
    # and the bound is not vacuous: a few ulps of the values it bounds
    rel = EX / np.maximum(np.abs(Xo), 1e-300)
    assert np.median(rel[np.abs(Xo) > 1e-3 * np.abs(Xo).max()]) < 200 * U32


def test_pattern_has_pairs_off_the_diagonal(case):
    s = case[0]
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    off = [p for p in range(len(s.colind)) if rows[p] != s.colind[p]
           and _pairs(s.rowptr, s.colind, rows[p], s.colind[p])]
    assert len(off) > 20


def _planted(s, X, D, Xo, defect):
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    bad = Xo.copy()
    for p in range(len(s.colind)):
        i, j = rows[p], s.colind[p]
        pr = _pairs(s.rowptr, s.colind, i, j)
        if not pr or j >= i:
            continue
        q, r = pr[0]
        if defect == "drop_pair":
            dS = X[q] @ X[r]
        elif defect == "transposed":
            dS = X[q] @ X[r] - X[q].T @ X[r]
        Sij = Xo[p] @ np.linalg.inv(D[j])
        bad[p] = (Sij + dS) @ D[j]
        return bad
    raise AssertionError("no L block with a pair")


@pytest.mark.parametrize("defect", ["drop_pair", "transposed"])
def test_planted_defects_fall_outside(case, defect):
    s, X, D, Xo, Do, EX, ED = case
    bad = _planted(s, X, D, Xo, defect)
    assert not _inside(np.abs(bad - Xo), EX, Xo)


def test_stale_dinv_falls_outside(case):
    """L updated with inv(U_jj) of the iterate before X^k (a stale input)."""
    s, X, D, Xo, Do, EX, ED = case
    Xp, Dp, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    Xs, _, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, X, Dp)
    assert not _inside(np.abs(Xs - Xo), EX, Xo)
