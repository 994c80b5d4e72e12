"""Entry-wise bounds of the FP32 rounding error of one block ILU sweep
(Eq. bilu / Eq. blockH) evaluated in FP32 from given factors, for the tests
that pin the FP32/BF16 build kernels against the FP64 oracle.

For the block (i, j) with np product pairs, S_ij = A_ij - sum L_ik U_kj is an
inner product of 4 np + 1 terms (A rounded to FP32 once, each product row 4
multiply-adds, one subtraction per pair) whose summation tree has depth at most
np + 5, so (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1)
    |S_fp32 - S| <= (np + 6) u (|A_ij| + (|L_s| |U_s|)_ij),   u = 2^-24,
|L_s| |U_s| being the product of the entry-wise absolute strictly lower and
strictly upper factors restricted to the pattern.  L_ij = S_ij Dinv_j adds
    E_S |Dinv_j| + 5 u |S| |Dinv_j|,
and Dinv_i = inv(U_ii) (refined to within 8 u max|Dinv_i| of the exact inverse
of the FP32 U_ii) moves by at most 1.1 |Dinv| E_U |Dinv| + 8 u max|Dinv_i|.
"""
import numpy as np
import scipy.sparse as sp

U32 = 2.0 ** -24
U16 = 2.0 ** -8


def _bsr(rowptr, colind, blocks, keep, n):
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    r, c, b = rows[keep], colind[keep], blocks[keep]
    ptr = np.concatenate([[0], np.cumsum(np.bincount(r, minlength=n))]).astype(np.int64)
    return sp.bsr_matrix((np.ascontiguousarray(b), c.astype(np.int64), ptr),
                         shape=(4 * n, 4 * n), blocksize=(4, 4))


def _blocks_at(M, rowptr, colind, n):
    """The 4x4 blocks of BSR matrix M at the pattern's positions (zero where M
    has no block)."""
    M = M.tobsr(blocksize=(4, 4))
    M.sort_indices()
    mrows = np.repeat(np.arange(n, dtype=np.int64), np.diff(M.indptr))
    mkey = mrows * n + M.indices
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    key = rows * n + colind
    out = np.zeros((len(colind), 4, 4))
    pos = np.searchsorted(mkey, key)
    ok = pos < len(mkey)
    ok[ok] = mkey[pos[ok]] == key[ok]
    out[ok] = M.data[pos[ok]]
    return out


def sweep_bound(s, X, D):
    """Entry-wise bounds of the FP32 rounding error of one sweep from (X, D)
    (FP64 arrays holding the stored factors): (E_X, E_D) as derived above."""
    n = s.n
    rows = np.repeat(np.arange(n), np.diff(s.rowptr))
    lo, up, dg = s.colind < rows, s.colind > rows, s.colind == rows
    Ls = _bsr(s.rowptr, s.colind, X, lo, n)
    Us = _bsr(s.rowptr, s.colind, X, up, n)
    absLU = _blocks_at(abs(Ls) @ abs(Us), s.rowptr, s.colind, n)
    S = s.vals - _blocks_at(Ls @ Us, s.rowptr, s.colind, n)
    ones = np.ones((len(s.colind), 4, 4))
    npairs = _blocks_at(_bsr(s.rowptr, s.colind, ones, lo, n) @ _bsr(s.rowptr, s.colind, ones, up, n),
                        s.rowptr, s.colind, n)[:, 0, 0] / 4.0
    ES = (npairs[:, None, None] + 6.0) * U32 * (np.abs(s.vals) + absLU)
    EX = ES.copy()
    Dj = np.abs(D[s.colind[lo]])
    EX[lo] = ES[lo] @ Dj + 5.0 * U32 * (np.abs(S[lo]) @ Dj)
    EU = ES[dg]                       # U_ii, in row order
    Da = np.abs(D)
    ED = 1.1 * (Da @ EU @ Da) + 8.0 * U32 * Da.max(axis=(1, 2))[:, None, None]
    return EX, ED
