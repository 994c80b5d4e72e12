"""The FP32/BF16 block work-item build sweeps pinned at FP32-arithmetic
tolerance against the oracle.

One synchronous sweep of Eq. (bilu) with FP32/BF16 factors
(k_build_blocks_sync) starts from an iterate (X^k, Dinv^k) that the test
exports from the GPU, and the oracle's FP64 sweep (orc_bilu_sync_sweep,
Eq. blockH) starts from the same exported values.  The two results differ only
by the GPU's FP32 rounding, which is bounded element by element:

* S_ij = A_ij - sum_{t} L_ik U_kj over the block's np product pairs.  The GPU
  rounds A to FP32 once, forms each 4x4 product row with 4 FP32 multiply-adds
  and subtracts it: an inner product of 4 np + 1 terms whose summation tree has
  depth at most np + 5.  The standard inner-product bound (Higham, Accuracy and
  Stability of Numerical Algorithms, Sec. 3.1) gives
      |S_gpu - S| <= (np + 6) u (|A_ij| + (|L_s| |U_s|)_ij)     (u = 2^-24)
  entry by entry, |L_s| |U_s| being the product of the entry-wise absolute
  values of the strictly lower and strictly upper factors restricted to the
  pattern (exactly the sum over the pairs of |L_ik| |U_kj|).  U blocks and the
  diagonal U_ii are S itself.
* L_ij = S_ij Dinv_j (4-term FP32 products with the same exported Dinv_j):
      |L_gpu - L| <= E_S |Dinv_j| + 5 u |S| |Dinv_j|.
* Dinv_i = inv(U_ii): the refined FP32 inverse is within 8 u max|Dinv_i| of
  the exact inverse of the GPU's U_ii, and inv(U_ii) moves by at most
  |Dinv_i| E_U |Dinv_i| to first order when U_ii moves by E_U:
      |Dinv_gpu - Dinv| <= 1.1 |Dinv| E_U |Dinv| + 8 u max|Dinv_i|.
* BF16 storage adds its unit roundoff 2^-8 times the stored value.

Every bound is written in the test; the test also reports the largest ratio of
the error to the bound.  A plausible defect anywhere in the sweep (a dropped or
doubled pair, a transposed product, the wrong Dinv, a stale input) moves the
result by O(|L||U|), far above a few ulps.

The asynchronous kernel (k_build_blocks_async) runs the same per-block
arithmetic in place; its results are not unique (Sec. 4.2), but after enough
sweeps it sits at the fixed point of the FP32 map, so one oracle sweep from its
exported factors must return them within a few times the same bound.
"""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle
from fp32_bounds import U16, U32, sweep_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1912_00539_gb300 as m
    return m


class Sys:
    """The pattern and values of a system (host arrays)."""

    def __init__(self, name, rowptr, colind, vals):
        self.name = name
        self.rowptr = np.ascontiguousarray(rowptr, np.int32)
        self.colind = np.ascontiguousarray(colind, np.int32)
        self.vals = np.ascontiguousarray(vals, np.float64)
        self.n = len(rowptr) - 1


def _sys(s):
    return Sys(s.name, s.rowptr, s.colind, s.vals)


def _mg_coarse_level(ab):
    """Level 1 of the aggregation hierarchy of the 64x64 workload: a coarse
    pattern with triangles (the general product-pair path of the build)."""
    import torch
    s = gen.workload("inviscid_64x64")
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    mg = ab.Multigrid(pat, torch.from_numpy(s.vals).cuda(), max_levels=2)
    lv = mg.level(1)
    torch.cuda.synchronize()
    return Sys("mg_level1_64x64", lv["rowptr"].cpu().numpy(), lv["colind"].cpu().numpy(),
               lv["vals"].cpu().numpy())


SYSTEMS = {
    "random_triangles": lambda ab: _sys(gen.random_pattern_system(150, 400, seed=4)),
    "full8": lambda ab: _sys(gen.random_pattern_system(8, 0, seed=5, structure="full")),
    "grid37x11_ragged": lambda ab: _sys(gen.small_system(37, 11, seed=2)),
    "inviscid_64x64": lambda ab: _sys(gen.workload("inviscid_64x64")),
    "mg_level1_64x64": _mg_coarse_level,
}


def _check(err, bound, floor, what):
    ratio = float((err / (bound + floor)).max())
    assert ratio <= 1.0, f"{what}: error / bound = {ratio:.3g}"
    return ratio


def _gpu(ab, s):
    import torch
    rp = torch.from_numpy(s.rowptr).cuda()
    ci = torch.from_numpy(s.colind).cuda()
    return ab.Pattern(rp, ci), torch.from_numpy(s.vals).cuda()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("k", [0, 2])
@pytest.mark.parametrize("which", list(SYSTEMS))
def test_fp32_sync_sweep_from_exported_iterate(ab, which, k, dtype):
    """GPU sweep k+1 (FP32 arithmetic) vs the oracle's FP64 sweep from the
    GPU's exported X^k, Dinv^k, within the derived bound."""
    s = SYSTEMS[which](ab)
    pat, A = _gpu(ab, s)
    fac = ab.Factors(pat, dtype)
    fac.build(A, k, mode="sync")
    Xk, Dk = (t.cpu().numpy() for t in fac.export())
    fac.build(A, 1, mode="sync", init="previous")
    X1, D1 = (t.cpu().numpy() for t in fac.export())
    Xo, Do, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, Xk, Dk)
    EX, ED = sweep_bound(s, Xk, Dk)
    if dtype == "bf16":   # the stored result is rounded to BF16 once more
        EX = EX + 1.01 * U16 * np.abs(X1)
        ED = ED + 1.01 * U16 * np.abs(D1)
    floor_x = 1e-14 * np.abs(Xo).max()
    floor_d = 1e-14 * np.abs(Do).max()
    rx = _check(np.abs(X1 - Xo), EX, floor_x, f"{which} X")
    rd = _check(np.abs(D1 - Do), ED, floor_d, f"{which} Dinv")
    print(f"{which} k={k} {dtype}: max error/bound X {rx:.3f}, Dinv {rd:.3f}")


@pytest.mark.parametrize("which", list(SYSTEMS))
def test_fp32_async_build_is_a_fixed_point_of_the_oracle_sweep(ab, which):
    """Enough asynchronous FP32 sweeps reach the fixed point of the FP32 map:
    one oracle sweep from the exported factors returns them within 4x the
    one-sweep bound (the last values each block read may differ from the final
    ones by one rounding-level update)."""
    s = SYSTEMS[which](ab)
    pat, A = _gpu(ab, s)
    fac = ab.Factors(pat, "f32")
    fac.build(A, min(2 * s.n + 4, 64), mode="async")
    X, D = (t.cpu().numpy() for t in fac.export())
    Xo, Do, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, X, D)
    EX, ED = sweep_bound(s, X, D)
    rx = _check(np.abs(X - Xo), 4.0 * EX, 1e-14 * np.abs(Xo).max(), f"{which} X")
    rd = _check(np.abs(D - Do), 4.0 * ED, 1e-14 * np.abs(Do).max(), f"{which} Dinv")
    print(f"{which} async: max error/(4 bound) X {rx:.3f}, Dinv {rd:.3f}")


@pytest.mark.slow
def test_fp32_sweeps_512x512_from_exported_iterate(ab):
    """The 524,288-cell workload in the benchmark's launch configuration: one
    synchronous FP32 sweep from the exported iterate after 2 sweeps, and the
    asynchronous build after 48 sweeps, both within the derived bound."""
    s = _sys(gen.workload("inviscid_512x512"))
    pat, A = _gpu(ab, s)
    fac = ab.Factors(pat, "f32")
    fac.build(A, 2, mode="sync")
    Xk, Dk = (t.cpu().numpy() for t in fac.export())
    fac.build(A, 1, mode="sync", init="previous")
    X1, D1 = (t.cpu().numpy() for t in fac.export())
    Xo, Do, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, Xk, Dk)
    EX, ED = sweep_bound(s, Xk, Dk)
    rx = _check(np.abs(X1 - Xo), EX, 1e-14 * np.abs(Xo).max(), "512x512 sync X")
    rd = _check(np.abs(D1 - Do), ED, 1e-14 * np.abs(Do).max(), "512x512 sync Dinv")
    fac.build(A, 48, mode="async")
    X, D = (t.cpu().numpy() for t in fac.export())
    Xo, Do, _ = oracle.bilu_sync_sweep(s.rowptr, s.colind, s.vals, X, D)
    EX, ED = sweep_bound(s, X, D)
    ra = _check(np.abs(X - Xo), 4.0 * EX, 1e-14 * np.abs(Xo).max(), "512x512 async X")
    rb = _check(np.abs(D - Do), 4.0 * ED, 1e-14 * np.abs(Do).max(), "512x512 async Dinv")
    print(f"512x512: sync X {rx:.3f} Dinv {rd:.3f}; async X {ra:.3f} Dinv {rb:.3f}")
