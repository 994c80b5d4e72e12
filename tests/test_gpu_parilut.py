"""Threshold block ILU on the GPU (through the C ABI) against the oracle.

* Final pattern (rowptr, colind): integer, compared exactly.  The selection
  compares squared block norms formed in the same order on both sides from
  factors that agree to rounding; with the generator's continuous values no two
  norms at a budget boundary are that close.
* Factors (X, Dinv) after FP64 synchronous sweeps: 1e-12 of the oracle's (the
  tolerance of the single-pattern FP64 sweeps).
* FGMRES with these factors: iteration count within 10% (at least 1) of the
  oracle's, true FP64 residual <= 1e-6.
"""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1912_00539_gb300 as m
    return m


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


class Dev:
    def __init__(self, ab, s):
        import torch
        self.s = s
        self.A = torch.from_numpy(np.ascontiguousarray(s.vals)).cuda()
        self.b = torch.from_numpy(np.ascontiguousarray(s.b)).cuda()
        self.pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())

    def vec(self):
        import torch
        return torch.zeros((self.s.n, 4), dtype=torch.float64, device="cuda")


SYSTEMS = {
    "grid6x5": lambda: gen.small_system(6, 5, seed=1),
    "grid37x11_ragged": lambda: gen.small_system(37, 11, seed=2),
    "random_triangles": lambda: gen.random_pattern_system(150, 400, seed=4),
    "aniso40x20": lambda: gen.small_system(40, 20, seed=3, cfl=1e4, wall_normal_scale=100.0),
    "inviscid_64x64": lambda: gen.workload("inviscid_64x64"),
}


@pytest.fixture(scope="module", params=list(SYSTEMS))
def dsys(request, ab):
    return Dev(ab, SYSTEMS[request.param]())


def _compare(ab, d, fill, iters, sweeps):
    s = d.s
    pat, fac = ab.parilut(d.pat, d.A, fill=fill, iters=iters, sweeps=sweeps)
    rp, ci, Xo, Do = oracle.parilut(s.rowptr, s.colind, s.vals, fill=fill, iters=iters,
                                    sweeps=sweeps)
    grp, gci = pat.arrays()
    assert np.array_equal(grp.cpu().numpy(), rp) and np.array_equal(gci.cpu().numpy(), ci)
    X, D = fac.export()
    assert _rel(X.cpu().numpy(), Xo) < 1e-12 and _rel(D.cpu().numpy(), Do) < 1e-12
    return pat, fac, (rp, ci, Xo, Do)


@pytest.mark.parametrize("fill,iters,sweeps", [(2.0, 3, 2), (1.0, 2, 1), (1.5, 1, 3)])
def test_parilut_matches_oracle(ab, dsys, fill, iters, sweeps):
    _compare(ab, dsys, fill, iters, sweeps)


def test_no_steps_is_block_ilu(ab, dsys):
    """iters = 0: block ILU(0) after `sweeps` synchronous sweeps on a copy of
    A's pattern, bit for bit the factors of abilu_build."""
    pat, fac = ab.parilut(dsys.pat, dsys.A, fill=2.0, iters=0, sweeps=3)
    assert pat.nnzb == dsys.pat.nnzb
    f2 = ab.Factors(dsys.pat, "f64")
    f2.build(dsys.A, 3, mode="sync")
    X1, D1 = fac.export()
    X2, D2 = f2.export()
    assert np.array_equal(X1.cpu().numpy(), X2.cpu().numpy())
    assert np.array_equal(D1.cpu().numpy(), D2.cpu().numpy())


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_fgmres_with_threshold_factors(ab, dsys, mode):
    s = dsys.s
    pat, fac, (rp, ci, Xo, Do) = _compare(ab, dsys, 2.0, 3, 2)
    x = dsys.vec()
    res = ab.fgmres_solve(dsys.pat, dsys.A, fac, dsys.b, x, restart=30, rtol=1e-6,
                          apply_sweeps_lower=3, apply_sweeps_upper=3, mode=mode, build=False,
                          max_iters=300)
    _, ro = oracle.fgmres_ilu_pattern(s.rowptr, s.colind, s.vals, rp, ci, Xo, Do, s.b, 3, 3,
                                      restart=30, max_iters=300)
    assert res.converged and ro.converged
    tol = max(1, ro.iters // 10)
    if mode == "sync":
        assert abs(res.iters - ro.iters) <= tol, (res.iters, ro.iters)
    else:   # in-place sweeps read newer values: never more than 10% above
        assert res.iters <= ro.iters + tol, (res.iters, ro.iters)
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6


def test_foreign_pattern_needs_no_build(ab):
    d = Dev(ab, gen.small_system(6, 5, seed=1))
    pat, fac = ab.parilut(d.pat, d.A)
    with pytest.raises(ab.AbiluError) as e:
        ab.fgmres_solve(d.pat, d.A, fac, d.b, d.vec(), build=True)
    assert e.value.status == 1


@pytest.mark.slow
def test_full_size_viscous(ab):
    """The 524,288-cell viscous-like workload: the final pattern (3.6 M blocks)
    and factors equal the oracle's, and FGMRES(50) with them converges with
    the oracle's iteration count."""
    s = gen.workload("viscous_1024x256_rcm")
    d = Dev(ab, s)
    pat, fac, (rp, ci, Xo, Do) = _compare(ab, d, 2.0, 3, 2)
    x = d.vec()
    res = ab.fgmres_solve(d.pat, d.A, fac, d.b, x, restart=50, rtol=1e-6, apply_sweeps_lower=6,
                          apply_sweeps_upper=6, mode="sync", build=False, max_iters=300)
    _, ro = oracle.fgmres_ilu_pattern(s.rowptr, s.colind, s.vals, rp, ci, Xo, Do, s.b, 6, 6,
                                      restart=50, max_iters=300)
    assert res.converged and abs(res.iters - ro.iters) <= max(1, ro.iters // 10)
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6


def test_block_diagonal_has_no_fill(ab):
    """Block-diagonal A: L U has no fill and no off-diagonal block to keep;
    the pattern stays the diagonal and the factors are the exact inverse."""
    s = gen.random_pattern_system(300, 0, seed=9, structure="diagonal")
    d = Dev(ab, s)
    pat, fac = ab.parilut(d.pat, d.A, fill=2.0, iters=2, sweeps=1)
    rp, ci = pat.arrays()
    assert np.array_equal(rp.cpu().numpy(), s.rowptr) and np.array_equal(ci.cpu().numpy(), s.colind)
    X, D = fac.export()
    assert _rel(D.cpu().numpy(), np.linalg.inv(s.vals)) < 1e-14


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-6), ("bf16", 8e-3)])
def test_narrow_storage_of_the_factors(ab, dsys, dtype, tol):
    """Factors computed in FP64 and stored in FP32 / BF16: the stored values
    are the oracle's rounded (unit roundoff 6e-8 / 3.9e-3 of the largest
    entry), and FGMRES with them converges like the FP64 ones (FP32: the
    oracle's iteration count within 10%, at least 1)."""
    s = dsys.s
    pat, fac = ab.parilut(dsys.pat, dsys.A, fill=2.0, iters=3, sweeps=2, dtype=dtype)
    rp, ci, Xo, Do = oracle.parilut(s.rowptr, s.colind, s.vals, fill=2.0, iters=3, sweeps=2)
    grp, gci = pat.arrays()
    assert np.array_equal(grp.cpu().numpy(), rp) and np.array_equal(gci.cpu().numpy(), ci)
    X, D = fac.export()
    assert _rel(X.cpu().numpy(), Xo) < tol and _rel(D.cpu().numpy(), Do) < tol
    x = dsys.vec()
    res = ab.fgmres_solve(dsys.pat, dsys.A, fac, dsys.b, x, restart=30, rtol=1e-6,
                          apply_sweeps_lower=3, apply_sweeps_upper=3, mode="sync", build=False,
                          max_iters=300)
    _, ro = oracle.fgmres_ilu_pattern(s.rowptr, s.colind, s.vals, rp, ci, Xo, Do, s.b, 3, 3,
                                      restart=30, max_iters=300)
    assert res.converged
    if dtype == "f32":
        assert abs(res.iters - ro.iters) <= max(1, ro.iters // 10), (res.iters, ro.iters)
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6
