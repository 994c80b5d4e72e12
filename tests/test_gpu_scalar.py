"""Parity of the scalar ILU(0) variant (Chow-Patel, Sec. 3.2) on the GPU with
the oracle's scalar functions, through the C ABI.  FP64: synchronous sweeps
and applications within 1e-12 of the oracle (the sums differ only in their
rounding order); asynchronous ones reach the fixed point / exact solve with
enough sweeps."""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "grid4x3": lambda: gen.small_system(4, 3, seed=1),
    "grid37x11_ragged": lambda: gen.small_system(37, 11, seed=2),
    "random_triangles": lambda: gen.random_pattern_system(150, 400, seed=4),
    "full8": lambda: gen.random_pattern_system(8, 0, seed=5, structure="full"),
    "inviscid_64x64": lambda: gen.workload("inviscid_64x64"),
}


@pytest.fixture(scope="module")
def ab():
    import torch
    assert torch.cuda.is_available()
    import paper_1912_00539_gb300 as m
    return m


@pytest.fixture(scope="module", params=list(SYSTEMS))
def dsys(request, ab):
    import torch
    s = SYSTEMS[request.param]()

    class D:
        pass
    d = D()
    d.s = s
    d.pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    d.A = torch.from_numpy(np.ascontiguousarray(s.vals)).cuda()
    d.b = torch.from_numpy(np.ascontiguousarray(s.b)).cuda()
    return d


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _vec(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("nsweeps", [0, 1, 2, 4])
def test_sync_build_matches_oracle(ab, dsys, nsweeps):
    s = dsys.s
    fac = ab.Factors(dsys.pat, "f64", scalar=True)
    fac.build(dsys.A, nsweeps, mode="sync")
    X, _ = fac.export()
    Xo, _ = oracle.silu_sync(s.rowptr, s.colind, s.vals, nsweeps)
    assert _rel(X.cpu().numpy(), Xo) < 1e-12


def test_sync_build_reaches_sequential(ab, dsys):
    s = dsys.s
    if s.n > 1000:
        pytest.skip("small systems")
    fac = ab.Factors(dsys.pat, "f64", scalar=True)
    fac.build(dsys.A, 4 * s.n + 8, mode="sync")
    X, _ = fac.export()
    Xs, _ = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    assert _rel(X.cpu().numpy(), Xs) < 1e-12


@pytest.mark.parametrize("nl,nu", [(1, 1), (2, 3), (4, 4), (0, 2), (3, 0)])
def test_sync_apply_matches_oracle(ab, dsys, nl, nu):
    s = dsys.s
    fac = ab.Factors(dsys.pat, "f64", scalar=True)
    fac.build(dsys.A, 3, mode="sync")
    X, _ = fac.export()
    r = np.random.default_rng(5).standard_normal((s.n, 4))
    z = _vec(np.ones((s.n, 4)))
    fac.apply(_vec(r), z, nl, nu, mode="sync")
    zo = oracle.silu_apply(s.rowptr, s.colind, X.cpu().numpy(), r, nl, nu)
    assert _rel(z.cpu().numpy(), zo) < 1e-12 if np.abs(zo).max() > 0 else not z.cpu().numpy().any()


def test_async_build_and_apply_reach_exact(ab, dsys):
    """The asynchronous iteration converges to the same fixed point; in-place
    triangular sweeps reach exact substitution."""
    s = dsys.s
    if s.n > 1000:
        pytest.skip("small systems")
    fac = ab.Factors(dsys.pat, "f64", scalar=True)
    fac.build(dsys.A, 4 * s.n + 8, mode="async")
    X, _ = fac.export()
    Xs, _ = oracle.silu0_seq(s.rowptr, s.colind, s.vals)
    assert _rel(X.cpu().numpy(), Xs) < 1e-12
    r = np.random.default_rng(6).standard_normal((s.n, 4))
    z = _vec(np.zeros((s.n, 4)))
    fac.apply(_vec(r), z, 4 * s.n + 1, 4 * s.n + 1, mode="async")
    zo = oracle.silu_apply(s.rowptr, s.colind, Xs, r, -1, -1)
    assert _rel(z.cpu().numpy(), zo) < 1e-12


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_fgmres_with_scalar_preconditioner(ab, dsys, mode):
    """Converges to 1e-6; sync FP64 takes the oracle's iteration count (the
    only differences are rounding order), async within +-10% (at least 1)."""
    import torch
    s = dsys.s
    fac = ab.Factors(dsys.pat, "f64", scalar=True)
    x = torch.zeros_like(dsys.b)
    res = ab.fgmres_solve(dsys.pat, dsys.A, fac, dsys.b, x, restart=30, rtol=1e-6,
                          build_sweeps=3, apply_sweeps_lower=3, apply_sweeps_upper=3, mode=mode)
    assert res.converged and res.rel_resid_true <= 1e-6
    Xo, _ = oracle.silu_sync(s.rowptr, s.colind, s.vals, 3)
    _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, None, s.b, 3, 3, restart=30, rtol=1e-6)
    if mode == "sync":
        assert res.iters == ro.iters, (res.iters, ro.iters)
    else:
        assert abs(res.iters - ro.iters) <= max(1, ro.iters // 10), (res.iters, ro.iters)
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(s.b)


def test_zero_pivot_counted_like_the_oracle(ab):
    import torch
    s = gen.small_system(3, 3, seed=8)
    vals = s.vals.copy()
    vals[s.rowptr[0], 0, 0] = 0.0
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    fac = ab.Factors(pat, "f64", scalar=True)
    fac.build(torch.from_numpy(vals).cuda(), 3, mode="sync")
    X, _ = fac.export()
    Xo, ns = oracle.silu_sync(s.rowptr, s.colind, vals, 3)
    assert ns > 0 and fac.singular_blocks() == ns
    assert _rel(X.cpu().numpy(), Xo) < 1e-12


def test_scalar_rejects_narrow_dtypes_and_diagnostics(ab, dsys):
    with pytest.raises(ab.AbiluError):
        ab.Factors(dsys.pat, "f32", scalar=True)
    fac = ab.Factors(dsys.pat, "f64", scalar=True)
    fac.build(dsys.A, 1)
    with pytest.raises(ab.AbiluError):
        fac.diagnostics(dsys.A)
