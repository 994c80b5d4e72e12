"""Dense numpy brute force used to pin the C oracle on tiny systems.

TEST INFRASTRUCTURE ONLY.  Written independently of ``abilu_oracle.c``: the
block ILU(0) here is the textbook IKJ elimination (Saad, Iterative Methods for
Sparse Linear Systems, Alg. 10.4, in block form) on a dense copy of A that
drops every update falling outside the block pattern S_B, with
``numpy.linalg.inv`` for the pivot blocks; solves use ``numpy.linalg.solve``.
"""
from __future__ import annotations

import numpy as np


def block_mask(rowptr, colind):
    n = len(rowptr) - 1
    m = np.zeros((n, n), bool)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    m[rows, colind] = True
    return m


def to_blocks(rowptr, colind, vals):
    """Dense (n, n, 4, 4) block array from BSR."""
    n = len(rowptr) - 1
    W = np.zeros((n, n, 4, 4))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    W[rows, colind] = np.asarray(vals).reshape(-1, 4, 4)
    return W


def blocks_to_dense(W):
    n = W.shape[0]
    return W.transpose(0, 2, 1, 3).reshape(4 * n, 4 * n)


def to_dense(rowptr, colind, vals):
    return blocks_to_dense(to_blocks(rowptr, colind, vals))


def bilu0_ikj(rowptr, colind, vals):
    """Block ILU(0) by masked IKJ elimination -> dense block arrays (L, U),
    L unit lower block triangular, U upper block triangular."""
    mask = block_mask(rowptr, colind)
    W = to_blocks(rowptr, colind, vals)
    n = W.shape[0]
    for i in range(n):
        for k in range(i):
            if not mask[i, k]:
                continue
            W[i, k] = W[i, k] @ np.linalg.inv(W[k, k])
            for j in range(k + 1, n):
                if mask[i, j]:
                    W[i, j] = W[i, j] - W[i, k] @ W[k, j]
    L = np.zeros_like(W)
    U = np.zeros_like(W)
    for i in range(n):
        L[i, i] = np.eye(4)
        for j in range(n):
            if j < i:
                L[i, j] = W[i, j]
            else:
                U[i, j] = W[i, j]
    return L, U


def factors_from_pattern_layout(rowptr, colind, X):
    """Dense block (L, U) from factors stored in A's pattern layout."""
    W = to_blocks(rowptr, colind, X)
    n = W.shape[0]
    L = np.zeros_like(W)
    U = np.zeros_like(W)
    for i in range(n):
        L[i, i] = np.eye(4)
        for j in range(n):
            if j < i:
                L[i, j] = W[i, j]
            else:
                U[i, j] = W[i, j]
    return L, U


def pattern_layout_from_dense(rowptr, colind, L, U):
    """Inverse of ``factors_from_pattern_layout`` restricted to the pattern."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    out = np.where((rows < colind)[:, None, None] | (rows == colind)[:, None, None],
                   U[rows, colind], L[rows, colind])
    return out


def lu_solve_dense(L, U, r):
    """(LU)^{-1} r with numpy.linalg.solve on the dense factors."""
    M = blocks_to_dense(L) @ blocks_to_dense(U)
    return np.linalg.solve(M, np.asarray(r).reshape(-1)).reshape(-1, 4)


def scalar_mask(rowptr, colind):
    """The scalar pattern S: every entry of every block of the block pattern."""
    return np.kron(block_mask(rowptr, colind), np.ones((4, 4), bool))


def silu0_ikj(rowptr, colind, vals):
    """Scalar ILU(0) by masked IKJ elimination (Saad, Algorithm 10.4) on the
    dense scalar matrix -> dense (L, U), L unit lower triangular."""
    mask = scalar_mask(rowptr, colind)
    W = to_dense(rowptr, colind, vals).copy()
    n = W.shape[0]
    for i in range(1, n):
        for k in range(i):
            if not mask[i, k]:
                continue
            W[i, k] = W[i, k] / W[k, k]
            for j in range(k + 1, n):
                if mask[i, j]:
                    W[i, j] = W[i, j] - W[i, k] * W[k, j]
    L = np.tril(W, -1) + np.eye(n)
    U = np.triu(W)
    return L, U


def scalar_factors_dense(rowptr, colind, X):
    """Dense (L, U) of scalar factors held in A's block layout."""
    D = to_dense(rowptr, colind, X)
    n = D.shape[0]
    return np.tril(D, -1) + np.eye(n), np.triu(D)
