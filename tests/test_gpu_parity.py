"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (max-norm error relative to the max-norm of the oracle's result):
* FP64 synchronous build, FP64 apply: 1e-12 (the sync GPU sweeps evaluate the
  same formulas in the same order; only FMA contraction and the adjugate vs
  Gauss-Jordan inversion differ, a few ulps per sweep).
* SpMV: 1e-14 (16 products per block row entry, FMA rounding only).
* FP32 arithmetic on factors that the test exports from the GPU: 2e-6
  (unit roundoff 6e-8 times the ~10-term sums and 4x4 products of a sweep
  chain).
* FP32 / BF16 factor storage against the FP64 oracle build: 1e-4 / 4e-2
  (storage unit roundoff 6e-8 / 3.9e-3 amplified by the sweeps).
Integer results (pattern counts, pair lists) are exact.
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
    """A system on the device with its pattern handle."""

    def __init__(self, ab, s):
        import torch
        self.s = s
        self.rowptr = torch.from_numpy(s.rowptr).cuda()
        self.colind = torch.from_numpy(s.colind).cuda()
        self.A = torch.from_numpy(np.ascontiguousarray(s.vals)).cuda()
        self.b = torch.from_numpy(np.ascontiguousarray(s.b)).cuda()
        self.pat = ab.Pattern(self.rowptr, self.colind)

    def vec(self, a=None):
        import torch
        if a is None:
            return torch.zeros((self.s.n, 4), dtype=torch.float64, device="cuda")
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def one_block_system():
    rowptr = np.array([0, 1], np.int32)
    colind = np.array([0], np.int32)
    vals = np.array([[[4.0, 1, 0, 0], [1, 5, 1, 0], [0, 1, 6, 1], [0, 0, 1, 7]]])
    b = np.array([[1.0, 2, 3, 4]])
    return gen.System("one_block", rowptr, colind, vals, b, np.arange(1), 1.0)


SYSTEMS = {
    "grid4x3": lambda: gen.small_system(4, 3, seed=1),
    "grid37x11_ragged": lambda: gen.small_system(37, 11, seed=2),      # 814 cells: ragged CTA tail
    "grid100x60": lambda: gen.small_system(100, 60, seed=3),           # 12,000 cells, many tiles
    "random_triangles": lambda: gen.random_pattern_system(150, 400, seed=4),
    "full8": lambda: gen.random_pattern_system(8, 0, seed=5, structure="full"),
    "one_block": one_block_system,
    "inviscid_64x64": lambda: gen.workload("inviscid_64x64"),
}


@pytest.fixture(scope="module", params=list(SYSTEMS))
def dsys(request, ab):
    return Dev(ab, SYSTEMS[request.param]())


# ------------------------------------------------------------------ pattern

def test_pattern_counts_exact(ab, dsys):
    s = dsys.s
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    nbr = [set(s.colind[s.rowptr[i]:s.rowptr[i + 1]]) for i in range(s.n)]
    npairs = 0
    for i in range(s.n):
        for j in s.colind[s.rowptr[i]:s.rowptr[i + 1]]:
            npairs += sum(1 for k in nbr[i] if k < min(i, j) and j in nbr[k])
    c = dsys.pat.counts()
    assert c["n"] == s.n and c["nnzb"] == s.nnzb
    assert c["nl"] == int(np.sum(rows > s.colind)) and c["nu"] == int(np.sum(rows < s.colind))
    assert c["npairs"] == npairs
    assert c["max_row"] == int(np.diff(s.rowptr).max())
    # work list: every L and diagonal block plus the U blocks with a product pair
    u_with_pairs = sum(1 for i in range(s.n) for j in s.colind[s.rowptr[i]:s.rowptr[i + 1]]
                       if j > i and any(k < i and j in nbr[k] for k in nbr[i]))
    assert c["nwork"] == c["nl"] + s.n + u_with_pairs


@pytest.mark.parametrize("bad", ["unsorted", "no_diag", "col_range", "rowptr"])
def test_malformed_pattern_rejected(ab, bad):
    import torch
    s = gen.small_system(3, 2, seed=6)
    rp, ci = s.rowptr.copy(), s.colind.copy()
    if bad == "unsorted":
        ci[[0, 1]] = ci[[1, 0]]
    elif bad == "no_diag":  # drop the diagonal block of row 2
        d = rp[2] + int(np.flatnonzero(ci[rp[2]:rp[3]] == 2)[0])
        ci = np.delete(ci, d)
        rp[3:] -= 1
    elif bad == "col_range":
        ci[-1] = s.n + 3
    else:
        rp[3] = rp[4] + 1
    with pytest.raises(ab.AbiluError) as e:
        ab.Pattern(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda())
    assert e.value.status == 1


# --------------------------------------------------------------------- SpMV

def test_spmv_parity(ab, dsys):
    s = dsys.s
    x = np.random.default_rng(11).standard_normal((s.n, 4))
    y_ref = oracle.spmv(s.rowptr, s.colind, s.vals, x)
    y = dsys.vec()
    ab.bsr_spmv(dsys.pat, dsys.A, dsys.vec(x), y)
    assert _rel(y.cpu().numpy(), y_ref) < 1e-14
    # y = 2 A x - 0.5 y0
    y0 = np.random.default_rng(12).standard_normal((s.n, 4))
    yt = dsys.vec(y0)
    ab.bsr_spmv(dsys.pat, dsys.A, dsys.vec(x), yt, alpha=2.0, beta=-0.5)
    assert _rel(yt.cpu().numpy(), 2 * y_ref - 0.5 * y0) < 1e-14


# -------------------------------------------------------------- build (sync)

@pytest.mark.parametrize("nsweeps", [0, 1, 2, 4])
def test_sync_build_f64_parity(ab, dsys, nsweeps):
    s = dsys.s
    fac = ab.Factors(dsys.pat, "f64")
    fac.build(dsys.A, nsweeps, mode="sync")
    X, D = fac.export()
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, nsweeps)
    assert _rel(X.cpu().numpy(), Xo) < 1e-12
    assert _rel(D.cpu().numpy(), Do) < 1e-12


def test_sync_build_converges_to_sequential(ab, dsys):
    s = dsys.s
    if s.n > 2000:
        pytest.skip("sweep count to the fixed point grows with the chain depth")
    fac = ab.Factors(dsys.pat, "f64")
    fac.build(dsys.A, 2 * s.n + 4, mode="sync")
    X, D = fac.export()
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    assert _rel(X.cpu().numpy(), Xs) < 1e-12 and _rel(D.cpu().numpy(), Ds) < 1e-12


def test_sync_build_bit_reproducible(ab, dsys):
    fac = ab.Factors(dsys.pat, "f32")
    fac.build(dsys.A, 3, mode="sync")
    X1, D1 = fac.export()
    fac.build(dsys.A, 3, mode="sync")
    X2, D2 = fac.export()
    assert (X1 == X2).all() and (D1 == D2).all()


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-4), ("bf16", 4e-2)])
def test_sync_build_narrow_storage(ab, dsys, dtype, tol):
    s = dsys.s
    fac = ab.Factors(dsys.pat, dtype)
    fac.build(dsys.A, 3, mode="sync")
    X, D = fac.export()
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 3)
    assert _rel(X.cpu().numpy(), Xo) < tol
    assert _rel(D.cpu().numpy(), Do) < tol


def test_warm_start_continues_the_iteration(ab, dsys):
    """init=previous continues from the stored factors: 2 + 2 sweeps = 4 sweeps."""
    s = dsys.s
    fac = ab.Factors(dsys.pat, "f64")
    fac.build(dsys.A, 2, mode="sync")
    fac.build(dsys.A, 2, mode="sync", init="previous")
    X, D = fac.export()
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 4)
    assert _rel(X.cpu().numpy(), Xo) < 1e-12 and _rel(D.cpu().numpy(), Do) < 1e-12


# -------------------------------------------------------------- apply (sync)

@pytest.mark.parametrize("nl,nu", [(0, 0), (1, 1), (1, 3), (2, 1), (2, 2), (3, 3), (4, 4), (5, 2)])
def test_sync_apply_f64_parity(ab, dsys, nl, nu):
    s = dsys.s
    fac = ab.Factors(dsys.pat, "f64")
    fac.build(dsys.A, 2, mode="sync")
    X, D = fac.export()
    r = np.random.default_rng(13).standard_normal((s.n, 4))
    z = dsys.vec()
    fac.apply(dsys.vec(r), z, nl, nu, mode="sync")
    z_ref = oracle.apply(s.rowptr, s.colind, X.cpu().numpy(), D.cpu().numpy(), r, nl, nu)
    if nu == 0:
        assert not z.cpu().numpy().any()
    else:
        assert _rel(z.cpu().numpy(), z_ref) < 1e-12


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("nl,nu", [(1, 1), (3, 3), (4, 4)])
def test_sync_apply_narrow_parity(ab, dsys, dtype, nl, nu):
    """FP32 arithmetic on the stored (narrow) factors vs FP64 on the same factors."""
    s = dsys.s
    fac = ab.Factors(dsys.pat, dtype)
    fac.build(dsys.A, 2, mode="sync")
    X, D = fac.export()
    r = np.random.default_rng(14).standard_normal((s.n, 4))
    z = dsys.vec()
    fac.apply(dsys.vec(r), z, nl, nu, mode="sync")
    z_ref = oracle.apply(s.rowptr, s.colind, X.cpu().numpy(), D.cpu().numpy(), r, nl, nu)
    assert _rel(z.cpu().numpy(), z_ref) < 2e-6


def test_sync_apply_exact_with_enough_sweeps(ab, dsys):
    """Jacobi block triangular sweeps are exact after chain-depth + 1 sweeps
    (Theorem of Sec. 4.1: at most n/b)."""
    s = dsys.s
    if s.n > 1000:
        pytest.skip("depth-bound sweep counts are for small systems")
    fac = ab.Factors(dsys.pat, "f64")
    fac.build(dsys.A, s.n + 2, mode="sync")
    X, D = fac.export()
    Xn, Dn = X.cpu().numpy(), D.cpu().numpy()
    r = np.random.default_rng(15).standard_normal((s.n, 4))
    z = dsys.vec()
    fac.apply(dsys.vec(r), z, s.n, s.n, mode="sync")
    y = oracle.lower_solve(s.rowptr, s.colind, Xn, r)
    z_ref = oracle.upper_solve(s.rowptr, s.colind, Xn, Dn, y)
    assert _rel(z.cpu().numpy(), z_ref) < 1e-12


# -------------------------------------------------------------------- async

def test_async_build_reaches_fixed_point(ab, dsys):
    """The asynchronous iteration converges to the unique fixed point (Sec.
    4.2): with enough sweeps it matches sequential BILU(0)."""
    s = dsys.s
    if s.n > 2000:
        pytest.skip("small systems only")
    fac = ab.Factors(dsys.pat, "f64")
    fac.build(dsys.A, 2 * s.n + 4, mode="async")
    X, D = fac.export()
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    assert _rel(X.cpu().numpy(), Xs) < 1e-12 and _rel(D.cpu().numpy(), Ds) < 1e-12


def test_async_build_residual_not_worse_than_sync(ab, dsys):
    """Async sweeps read newer values than Jacobi sweeps; over 10 runs the
    ILU fixed-point residual after k sweeps stays within the sync one."""
    s = dsys.s
    k = 3
    Xsync, _, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, k)
    r_sync = oracle.ilu_residual_l1(s.rowptr, s.colind, s.vals, Xsync)
    res = []
    fac = ab.Factors(dsys.pat, "f64")
    for _ in range(10):
        fac.build(dsys.A, k, mode="async")
        X, _ = fac.export()
        res.append(oracle.ilu_residual_l1(s.rowptr, s.colind, s.vals, X.cpu().numpy()))
    assert np.mean(res) <= 1.0 * r_sync + 1e-12 * max(r_sync, 1.0)


def test_async_apply_exact_with_enough_sweeps(ab, dsys):
    s = dsys.s
    if s.n > 1000:
        pytest.skip("small systems only")
    fac = ab.Factors(dsys.pat, "f64")
    fac.build(dsys.A, 3, mode="sync")
    X, D = fac.export()
    Xn, Dn = X.cpu().numpy(), D.cpu().numpy()
    r = np.random.default_rng(16).standard_normal((s.n, 4))
    z = dsys.vec()
    fac.apply(dsys.vec(r), z, s.n + 1, s.n + 1, mode="async")
    y = oracle.lower_solve(s.rowptr, s.colind, Xn, r)
    z_ref = oracle.upper_solve(s.rowptr, s.colind, Xn, Dn, y)
    assert _rel(z.cpu().numpy(), z_ref) < 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_async_apply_first_updates(ab, dsys, dtype):
    """The asynchronous application starts with the first update of every
    unknown read from the zero guesses (y = r, x^1 = Dinv r): with one sweep
    per factor it is that update exactly, the synchronous result bit for bit;
    with no lower or no upper sweep the result is zero.  Against the oracle's
    sweeps on the exported factors: z = Dinv r."""
    s = dsys.s
    fac = ab.Factors(dsys.pat, dtype)
    fac.build(dsys.A, 2, mode="sync")
    r = np.random.default_rng(17).standard_normal((s.n, 4))
    za, zs = dsys.vec(), dsys.vec()
    fac.apply(dsys.vec(r), za, 1, 1, mode="async")
    fac.apply(dsys.vec(r), zs, 1, 1, mode="sync")
    np.testing.assert_array_equal(za.cpu().numpy(), zs.cpu().numpy())
    if dtype == "f64":
        X, D = fac.export()
        z_ref = oracle.apply(s.rowptr, s.colind, X.cpu().numpy(), D.cpu().numpy(), r, 1, 1)
        assert _rel(za.cpu().numpy(), z_ref) < 1e-14
    for nl, nu in ((0, 2), (2, 0)):
        z = dsys.vec(np.ones((s.n, 4)))
        fac.apply(dsys.vec(r), z, nl, nu, mode="async")
        assert not z.cpu().numpy().any()


# ------------------------------------------------------------------- FGMRES

@pytest.mark.parametrize("dtype,mode", [("f64", "sync"), ("f32", "sync"), ("f32", "async"),
                                        ("bf16", "sync"), ("f64", "async")])
def test_fgmres_matches_oracle(ab, dsys, dtype, mode):
    s = dsys.s
    nb, na = 4, 3
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, nb)
    xo, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, na, na, restart=30,
                           rtol=1e-6)
    fac = ab.Factors(dsys.pat, dtype)
    x = dsys.vec()
    res = ab.fgmres_solve(dsys.pat, dsys.A, fac, dsys.b, x, restart=30, rtol=1e-6,
                          build_sweeps=nb, apply_sweeps_lower=na, apply_sweeps_upper=na,
                          mode=mode)
    assert res.converged and res.rel_resid_true <= 1e-6
    xn = x.cpu().numpy()
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, xn)
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6
    if dtype == "bf16":  # optional narrow variant: must converge, count is reported only
        assert res.iters <= 2 * ro.iters + 2
        return
    slack = max(1, int(np.ceil(0.1 * ro.iters)))
    assert abs(res.iters - ro.iters) <= slack, (res.iters, ro.iters)
    if dtype == "f64" and mode == "sync":
        assert res.iters == ro.iters


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("nl,nu", [(1, 1), (1, 3), (2, 1), (2, 3), (4, 4)])
def test_fgmres_async_application_starts(ab, dsys, dtype, nl, nu):
    """An asynchronous application starts from y = b and zeroed ticket counters:
    with one lower update its own start kernel does that (and forms x^1);
    with two or more, inside FGMRES, the kernels that write the FP32
    right-hand side do it.  On the same factors, both converge like the
    oracle's FGMRES with the same sweep counts (iterations within 10%), and
    the solution is checked with the oracle's SpMV."""
    s = dsys.s
    fac = ab.Factors(dsys.pat, dtype)
    fac.build(dsys.A, 4, mode="sync")
    X, D = fac.export()    # the oracle's FGMRES runs on the same (rounded) factors
    _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, X.cpu().numpy(), D.cpu().numpy(), s.b,
                          nl, nu, restart=30, rtol=1e-6)
    x = dsys.vec()
    res = ab.fgmres_solve(dsys.pat, dsys.A, fac, dsys.b, x, restart=30, rtol=1e-6,
                          apply_sweeps_lower=nl, apply_sweeps_upper=nu, mode="async", build=False)
    assert res.converged and res.rel_resid_true <= 1e-6
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6
    if dtype == "bf16":
        assert res.iters <= 2 * ro.iters + 2
        return
    slack = max(1, int(np.ceil(0.1 * ro.iters)))
    assert abs(res.iters - ro.iters) <= slack, (res.iters, ro.iters)


def test_fgmres_sync_bit_reproducible(ab):
    d = Dev(ab, gen.small_system(30, 20, seed=7))
    fac = ab.Factors(d.pat, "f32")
    xs = []
    for _ in range(2):
        x = d.vec()
        ab.fgmres_solve(d.pat, d.A, fac, d.b, x, build_sweeps=3, mode="sync")
        xs.append(x.cpu().numpy())
    np.testing.assert_array_equal(xs[0], xs[1])


@pytest.mark.parametrize("rtol", [1e-8, 1e-10])
@pytest.mark.parametrize("dtype,mode", [("f64", "sync"), ("f32", "sync"), ("f32", "async")])
def test_fgmres_tight_tolerances(ab, dsys, rtol, dtype, mode):
    """Below rtol 1e-7 the Arnoldi step forms h_{j+1,j} as the explicit norm
    of the updated w: the iteration count stays within 10% of the oracle's
    (modified Gram-Schmidt, same sweeps) and the true residual reaches rtol.
    The single-reduction form's sqrt(||w||^2 - sum h^2) loses accuracy as the
    classical basis loses orthogonality (a 96-cell system took 21 iterations
    against the oracle's 8 at 1e-8 with it)."""
    s = dsys.s
    nb, na = 4, 3
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, nb)
    _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, na, na, restart=30, rtol=rtol)
    fac = ab.Factors(dsys.pat, dtype)
    x = dsys.vec()
    res = ab.fgmres_solve(dsys.pat, dsys.A, fac, dsys.b, x, restart=30, rtol=rtol,
                          build_sweeps=nb, apply_sweeps_lower=na, apply_sweeps_upper=na,
                          mode=mode)
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
    assert res.converged and np.linalg.norm(r) / np.linalg.norm(s.b) <= rtol * 1.001
    if dtype == "f32" and (rtol < 1e-9 or mode == "async"):
        # FP32 factors: the preconditioner's rounding (and in asynchronous
        # mode its schedule), not the Arnoldi step, sets how far the count
        # may drift
        assert res.iters <= 2 * ro.iters + 2, (res.iters, ro.iters)
        return
    slack = max(1, int(np.ceil(0.1 * ro.iters)))
    assert abs(res.iters - ro.iters) <= slack, (res.iters, ro.iters)


def test_fgmres_restarts_and_reorth(ab):
    s = gen.small_system(12, 10, seed=8, cfl=1.0)
    d = Dev(ab, s)
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    xo, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, 1, 1, restart=4,
                           max_iters=500, rtol=1e-8)
    for reorth in (False, True):
        fac = ab.Factors(d.pat, "f64")
        x = d.vec()
        res = ab.fgmres_solve(d.pat, d.A, fac, d.b, x, restart=4, max_iters=500, rtol=1e-8,
                              build_sweeps=1, apply_sweeps_lower=1, apply_sweeps_upper=1,
                              mode="sync", reorth=reorth)
        assert res.converged and res.restarts >= 2
        assert abs(res.iters - ro.iters) <= max(2, ro.iters // 10), (res.iters, ro.iters)


@pytest.mark.parametrize("form", ["single", "classical", "cgs2"])
@pytest.mark.parametrize("nx,ny", [(30, 20), (240, 160)])
def test_fgmres_steps_past_the_fused_width(ab, form, nx, ny):
    """Cycles longer than five Arnoldi steps: every step forms w = A z_j with
    the first pass's dot products (and ||w||^2 in the single-reduction form)
    in one kernel; the first three basis vectors are dotted in the product's
    own pass, wider steps re-read w for the tiles past the third.  In FP64 the
    whole cycle follows the oracle's (modified Gram-Schmidt) iteration count
    in each Gram-Schmidt form: rtol 1e-6 takes the single-reduction step, 1e-8
    the classical one with the explicit norm, reorth CGS2.  The 76,800-row
    system gives each thread of the fused kernel three rows of its grid stride
    and crosses a restart at 30."""
    s = gen.small_system(nx, ny, seed=3, cfl=1e4)
    d = Dev(ab, s)
    rtol = 1e-6 if form == "single" else 1e-8
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, 1, 1, restart=30, rtol=rtol)
    assert ro.iters > 5
    fac = ab.Factors(d.pat, "f64")
    x = d.vec()
    res = ab.fgmres_solve(d.pat, d.A, fac, d.b, x, restart=30, rtol=rtol, build_sweeps=1,
                          apply_sweeps_lower=1, apply_sweeps_upper=1, mode="sync",
                          reorth=form == "cgs2")
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
    assert res.converged and np.linalg.norm(r) / np.linalg.norm(s.b) <= rtol * 1.001
    assert abs(res.iters - ro.iters) <= max(1, ro.iters // 10), (res.iters, ro.iters)


XERR_SYSTEMS = {
    "grid30x20_cfl1e4": lambda: gen.small_system(30, 20, seed=3, cfl=1e4),
    "grid240x160_cfl1e4": lambda: gen.small_system(240, 160, seed=3, cfl=1e4),   # 76,800 rows
    "inviscid_64x64": lambda: gen.workload("inviscid_64x64"),
    "random_triangles": lambda: gen.random_pattern_system(150, 400, seed=4),
    "grid37x11_ragged": lambda: gen.small_system(37, 11, seed=2),
}


@pytest.mark.parametrize("form", ["single", "classical", "cgs2"])
@pytest.mark.parametrize("name", list(XERR_SYSTEMS))
def test_fgmres_fp64_solution_equals_oracle(ab, name, form):
    """The FP64 synchronous solve and the oracle's FGMRES (modified
    Gram-Schmidt) produce the same iterates in exact arithmetic, whichever
    Gram-Schmidt form the GPU takes (single reduction at rtol 1e-6, classical
    with the explicit norm at 1e-8, CGS2): they stop at the same step and their
    solutions differ by rounding only.  Measured 8.5e-16 to 2.1e-14 relative
    (2-norm) over these systems, 10 to 20 iterations, so every width of the
    fused product-and-dots kernel runs; the bound 1e-11 leaves three orders of
    magnitude for rounding growth, while a wrong term of any dot product,
    norm or Givens rotation moves x in its leading digits."""
    s = XERR_SYSTEMS[name]()
    d = Dev(ab, s)
    rtol = 1e-6 if form == "single" else 1e-8
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 2)
    xo, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, 1, 1, restart=30, rtol=rtol)
    fac = ab.Factors(d.pat, "f64")
    x = d.vec()
    res = ab.fgmres_solve(d.pat, d.A, fac, d.b, x, restart=30, rtol=rtol, build_sweeps=2,
                          apply_sweeps_lower=1, apply_sweeps_upper=1, mode="sync",
                          reorth=form == "cgs2")
    assert res.converged and res.iters == ro.iters, (res.iters, ro.iters)
    xn = x.cpu().numpy()
    assert np.linalg.norm(xn - xo) / np.linalg.norm(xo) < 1e-11


def test_fgmres_max_iters_reports_noconv(ab):
    d = Dev(ab, gen.small_system(12, 10, seed=9, cfl=1.0))
    fac = ab.Factors(d.pat, "f64")
    x = d.vec()
    res = ab.fgmres_solve(d.pat, d.A, fac, d.b, x, restart=5, max_iters=3, rtol=1e-14,
                          build_sweeps=1, apply_sweeps_lower=1, apply_sweeps_upper=1, mode="sync")
    assert not res.converged and res.status == 4 and res.iters == 3


def test_fgmres_zero_rhs(ab):
    d = Dev(ab, gen.small_system(5, 5, seed=10))
    fac = ab.Factors(d.pat, "f64")
    x = d.vec(np.ones((d.s.n, 4)))
    res = ab.fgmres_solve(d.pat, d.A, fac, d.vec(), x, mode="sync")
    assert res.converged and res.iters == 0 and not x.cpu().numpy().any()


def test_singular_block_is_replaced_and_counted(ab):
    s = gen.small_system(4, 4, seed=11)
    vals = s.vals.copy()
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    d0 = np.flatnonzero((rows == 5) & (s.colind == 5))[0]
    vals[d0] = 0.0
    s2 = gen.System("sing", s.rowptr, s.colind, vals, s.b, s.perm, s.cfl)
    d = Dev(ab, s2)
    fac = ab.Factors(d.pat, "f64")
    fac.build(d.A, 0, mode="sync")
    assert fac.singular_blocks() == 1
    X, D = fac.export()
    np.testing.assert_array_equal(D.cpu().numpy()[5], np.eye(4))
    _, Do, ns = oracle.bilu_init(s2.rowptr, s2.colind, s2.vals)
    assert ns == 1 and _rel(D.cpu().numpy(), Do) < 1e-12


# ------------------------------------------------------------ full size

@pytest.mark.slow
def test_full_size_512x512_parity(ab):
    """The 512x512 workload at its solver settings: SpMV and one FP64 build
    sweep compared element by element; the FP32 solve (the benchmark's launch
    configuration) converges with iteration count within 10% of the FP64
    oracle's and a true FP64 residual below 1e-6."""
    s = gen.workload("inviscid_512x512")
    d = Dev(ab, s)
    x = np.random.default_rng(17).standard_normal((s.n, 4))
    y = d.vec()
    ab.bsr_spmv(d.pat, d.A, d.vec(x), y)
    assert _rel(y.cpu().numpy(), oracle.spmv(s.rowptr, s.colind, s.vals, x)) < 1e-14
    fac = ab.Factors(d.pat, "f64")
    fac.build(d.A, 1, mode="sync")
    X, D = fac.export()
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    assert _rel(X.cpu().numpy(), Xo) < 1e-12 and _rel(D.cpu().numpy(), Do) < 1e-12
    Xo6, Do6, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 6)
    _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo6, Do6, s.b, 4, 4, restart=30, rtol=1e-6)
    for mode in ("sync", "async"):
        f32 = ab.Factors(d.pat, "f32")
        xs = d.vec()
        res = ab.fgmres_solve(d.pat, d.A, f32, d.b, xs, restart=30, rtol=1e-6, build_sweeps=6,
                              apply_sweeps_lower=4, apply_sweeps_upper=4, mode=mode)
        assert res.converged and res.rel_resid_true <= 1e-6
        assert abs(res.iters - ro.iters) <= max(1, ro.iters // 10), (mode, res.iters, ro.iters)
        xn = xs.cpu().numpy()
        r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, xn)
        assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6


@pytest.mark.slow
def test_full_size_512x512_fp32_build_sweeps(ab):
    """FP32 factors at 512x512 (the benchmark's launch configuration of the
    block work-item sweeps): 3 synchronous sweeps match the oracle's 3 FP64
    sweeps within the FP32 storage tolerance;
    6 asynchronous sweeps leave an ILU fixed-point residual no larger than 6
    synchronous ones (they read newer values); 24 sweeps of either mode reach
    sequential BILU(0) (the unique fixed point, Sec. 4.2) within the FP32
    storage tolerance."""
    s = gen.workload("inviscid_512x512")
    d = Dev(ab, s)
    f32 = ab.Factors(d.pat, "f32")
    f32.build(d.A, 3, mode="sync")
    X, D = f32.export()
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 3)
    assert _rel(X.cpu().numpy(), Xo) < 1e-4 and _rel(D.cpu().numpy(), Do) < 1e-4
    Xo6, _, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 6)
    r_sync = oracle.ilu_residual_l1(s.rowptr, s.colind, s.vals, Xo6)
    f32.build(d.A, 6, mode="async")
    X, _ = f32.export()
    r_async = oracle.ilu_residual_l1(s.rowptr, s.colind, s.vals, X.cpu().numpy())
    assert r_async <= r_sync, (r_async, r_sync)
    # the default tickets (two 64-block sub-chunks half the list apart): the
    # blocks in flight span about 389 k consecutive work blocks in each half
    # of the list, so more of the rows a block reads are already updated in
    # the current sweep; measured 4.9-5.0 over runs, against 44 for tickets of
    # 128 consecutive blocks (a 778 k span)
    assert r_async < 20.0, r_async
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    for mode in ("sync", "async"):
        f32.build(d.A, 24, mode=mode)
        X, D = f32.export()
        assert _rel(X.cpu().numpy(), Xs) < 1e-4 and _rel(D.cpu().numpy(), Ds) < 1e-4, mode


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_refined_fp32_inverse_is_fp32_accurate(ab, dsys, mode):
    """FP32 factors: Dinv_i (FP32 adjugate + one error-free Newton step) equals
    the FP64 inverse of the stored FP32 U_ii to a few FP32 ulps."""
    s = dsys.s
    fac = ab.Factors(dsys.pat, "f32")
    fac.build(dsys.A, 3, mode=mode)
    X, D = fac.export()
    X, D = X.cpu().numpy(), D.cpu().numpy()
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    Uii = X[rows == s.colind]
    ref = np.linalg.inv(Uii)
    err = np.abs(D - ref).max(axis=(1, 2)) / np.abs(ref).max(axis=(1, 2))
    assert err.max() < 8 * 2.0 ** -24, err.max()


def test_fp64_to_fp32_rounding_is_exact(ab):
    """FP32 factors from 0 sweeps hold float32(A) in every L, U and U_ii block;
    the FP64->FP32 rounding (integer instructions on the GPU) must equal
    numpy's round-to-nearest-even bit for bit, ties, subnormals and extremes
    included."""
    s = gen.small_system(12, 9, seed=21)
    vals = s.vals.copy()
    rng = np.random.default_rng(22)
    special = np.array([1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, -(1 + 2.0 ** -24), 1 - 2.0 ** -25,
                        2.0 ** -130, -2.0 ** -140, 1e-300, 3.4e38, -3.3e38, 0.0, -0.0,
                        1.5 * 2.0 ** -126, 2.0 ** 127 * (2 - 2.0 ** -23),
                        np.nextafter(1.0, 2.0), 0.1, 1.0 / 3.0])
    # the bottom of the subnormal range (ties at 2^-150 and 3 * 2^-150), a
    # subnormal that rounds up into the smallest normal, overflow, Inf, NaN
    special = np.concatenate([special, [
        2.0 ** -150, 2.0 ** -150 * (1 + 2.0 ** -20), 3 * 2.0 ** -150, 2.0 ** -151,
        2.0 ** -126 * (1 - 2.0 ** -25), -2.0 ** -126 * (1 - 2.0 ** -30),
        3.5e38, -1e39, 2.0 ** 128 * (1 - 2.0 ** -25), np.inf, -np.inf, np.nan]])
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    offdiag = np.flatnonzero(rows != s.colind)          # non-finite values stay off U_ii
    entries = (offdiag[:, None] * 16 + np.arange(16)).reshape(-1)
    idx = rng.choice(entries, size=len(special) + 16 + 900, replace=False)
    flat = vals.reshape(-1)
    flat[idx[:len(special)]] = special
    # random doubles sitting exactly on float32 ties
    t = rng.standard_normal(900).astype(np.float32).astype(np.float64)
    ulp = np.abs(np.spacing(t.astype(np.float32)).astype(np.float64))
    flat[idx[len(special):len(special) + 900]] = t + 0.5 * ulp
    d = Dev(ab, gen.System("ties", s.rowptr, s.colind, vals, s.b, s.perm, s.cfl))
    fac = ab.Factors(d.pat, "f32")
    fac.build(d.A, 0, mode="sync")
    X, _ = fac.export()
    with np.errstate(over="ignore"):
        ref = vals.astype(np.float32).astype(np.float64)
    got = X.cpu().numpy()
    np.testing.assert_array_equal(got.view(np.int64), ref.view(np.int64))


def test_integer_fp32_conversion_is_exact(ab):
    """abilu_to_f32 (the integer-only conversion of the FGMRES normalisation)
    equals numpy's FP64 -> FP32 round to nearest even bit for bit: normal
    values, ties, subnormal results and their rounding into the smallest
    normal, the bottom of the subnormal range, overflow, Inf, NaN, zeros."""
    import torch
    rng = np.random.default_rng(23)
    x = rng.standard_normal(200000) * 10.0 ** rng.uniform(-48, 40, 200000)
    t = rng.standard_normal(20000).astype(np.float32).astype(np.float64)
    ties = t + 0.5 * np.abs(np.spacing(t.astype(np.float32)).astype(np.float64))
    sub = rng.integers(1, 2 ** 23, 20000) * 2.0 ** -149 + rng.choice([0.5, 0.25, 0.75], 20000) * 2.0 ** -149
    special = np.array([0.0, -0.0, 2.0 ** -150, 3 * 2.0 ** -150, 2.0 ** -151, 2.0 ** -1074,
                        2.0 ** -126 * (1 - 2.0 ** -25), 2.0 ** -126 * (1 - 2.0 ** -24),
                        3.4028234663852886e38, 2.0 ** 128 * (1 - 2.0 ** -25), 2.0 ** 128 * (1 - 2.0 ** -24),
                        1e39, -1e300, np.inf, -np.inf, np.nan, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24])
    allv = np.concatenate([x, ties, sub, -sub, special])
    d = torch.from_numpy(allv).cuda()
    out = torch.empty(allv.size, dtype=torch.float32, device="cuda")
    ab.to_f32(d, out)
    with np.errstate(over="ignore"):
        ref = allv.astype(np.float32)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_zero_guess_equals_explicit_zero_start(ab):
    """zero_guess overwrites x and starts from r0 = b; in synchronous mode the
    result is bit for bit that of an explicit x0 = 0 (A 0 = 0 exactly)."""
    import torch
    d = Dev(ab, gen.small_system(20, 15, seed=12))
    fac = ab.Factors(d.pat, "f32")
    x0 = d.vec()
    r0 = ab.fgmres_solve(d.pat, d.A, fac, d.b, x0, build_sweeps=3, mode="sync")
    x1 = d.vec(np.full((d.s.n, 4), 7.0))
    r1 = ab.fgmres_solve(d.pat, d.A, fac, d.b, x1, build_sweeps=3, mode="sync", zero_guess=True)
    assert r0.iters == r1.iters
    assert torch.equal(x0, x1)


@pytest.mark.parametrize("dtype,mode", [("f64", "sync"), ("f64", "async"), ("f32", "sync"),
                                        ("f32", "async"), ("bf16", "sync")])
def test_build_timing_events(ab, dtype, mode):
    """Build timing (abilu_factors_timing / abilu_factors_sweep_time): no time
    before a timed build or after timing is switched off; a timed build, alone
    or inside fgmres_solve, gives a positive device time; a synchronous build
    with timing on gives bit for bit the factors of one without."""
    import torch
    d = Dev(ab, gen.small_system(37, 11, seed=2))
    f1, f2 = ab.Factors(d.pat, dtype), ab.Factors(d.pat, dtype)
    with pytest.raises(ab.AbiluError):
        f1.sweep_ms()
    f1.timing(True)
    with pytest.raises(ab.AbiluError):
        f1.sweep_ms()
    f1.build(d.A, 3, mode)
    f2.build(d.A, 3, mode)
    assert f1.sweep_ms() > 0.0
    if mode == "sync":
        X1, D1 = f1.export()
        X2, D2 = f2.export()
        assert torch.equal(X1, X2) and torch.equal(D1, D2)
    f1.timing(True)   # re-enabling forgets the last time
    with pytest.raises(ab.AbiluError):
        f1.sweep_ms()
    res = ab.fgmres_solve(d.pat, d.A, f1, d.b, d.vec(), build_sweeps=2, mode=mode)
    assert res.converged and f1.sweep_ms() > 0.0
    f1.timing(False)
    with pytest.raises(ab.AbiluError):
        f1.sweep_ms()


@pytest.mark.parametrize("dtype,nsweeps", [("f64", 0), ("f64", 3), ("f32", 3)])
def test_diagnostics_match_oracle(ab, dsys, dtype, nsweeps):
    """GPU diagnostics (Sec. 6.2 quantities) equal the oracle's evaluated on the
    same (exported) factors."""
    s = dsys.s
    fac = ab.Factors(dsys.pat, dtype)
    fac.build(dsys.A, nsweeps, mode="sync")
    X, D = fac.export()
    Xn, Dn = X.cpu().numpy(), D.cpu().numpy()
    g = fac.diagnostics(dsys.A)
    r_ref = oracle.ilu_residual_l1(s.rowptr, s.colind, s.vals, Xn)
    d_ref = oracle.lu_defect_max(s.rowptr, s.colind, s.vals, Xn)
    ln, un = oracle.jacobi_norms(s.rowptr, s.colind, Xn, Dn)
    scale = np.abs(s.vals).max()
    assert abs(g["ilu_residual_l1"] - r_ref) <= 1e-9 * max(r_ref, 1.0) + 1e-9 * scale
    assert abs(g["lu_defect_max"] - d_ref) <= 1e-11 * scale
    assert abs(g["jacobi_norm_L"] - ln) <= 1e-12 * max(ln, 1.0)
    assert abs(g["jacobi_norm_U"] - un) <= 1e-10 * max(un, 1.0)


@pytest.mark.slow
@pytest.mark.parametrize("order", ["rcm", "line"])
def test_full_size_viscous_parity(ab, order):
    """The viscous-like 1024x256 workload (CFL 1e4, wall-normal coupling x100)
    in both orderings at its solver settings (8 build, 6+6 apply sweeps,
    FGMRES(50)): SpMV and one FP64 synchronous build sweep element by element
    (each inverse diagonal block to 64 u times its condition number: the two
    sides invert by different, equally valid methods);
    FP32-factor solves converge to a true FP64 residual <= 1e-6 with the FP64
    oracle's iteration count within 10% (synchronous) or at most 10% above it
    (asynchronous: newer values, the build nearer its fixed point)."""
    name = f"viscous_1024x256_{order}"
    s = gen.workload(name)
    st = gen.SOLVER_SETTINGS[name]
    d = Dev(ab, s)
    x = np.random.default_rng(19).standard_normal((s.n, 4))
    y = d.vec()
    ab.bsr_spmv(d.pat, d.A, d.vec(x), y)
    assert _rel(y.cpu().numpy(), oracle.spmv(s.rowptr, s.colind, s.vals, x)) < 1e-14
    fac = ab.Factors(d.pat, "f64")
    fac.build(d.A, 1, mode="sync")
    X, D = fac.export()
    Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 1)
    assert _rel(X.cpu().numpy(), Xo) < 1e-12
    # U_jj here reaches cond 9e6: two exact-arithmetic-equivalent inversions
    # (the GPU's adjugate, the oracle's Gauss-Jordan) differ by up to cond(U_jj)
    # units in the last place, so each inverse is held to 64 u cond(U_jj)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    cond = np.linalg.cond(Xo[rows == s.colind])
    err = np.abs(D.cpu().numpy() - Do).max(axis=(1, 2)) / np.abs(Do).max(axis=(1, 2))
    assert np.all(err <= 64 * 2.0 ** -53 * cond), float((err / cond).max())
    nb, na, m = st["build_sweeps"], st["apply_sweeps"], st["restart"]
    Xn, Dn, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, nb)
    _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xn, Dn, s.b, na, na, restart=m, rtol=1e-6)
    assert ro.converged
    for mode in ("sync", "async"):
        f32 = ab.Factors(d.pat, "f32")
        xs = d.vec()
        res = ab.fgmres_solve(d.pat, d.A, f32, d.b, xs, restart=m, rtol=1e-6, build_sweeps=nb,
                              apply_sweeps_lower=na, apply_sweeps_upper=na, mode=mode)
        assert res.converged and res.rel_resid_true <= 1e-6
        tol = max(1, ro.iters // 10)
        if mode == "sync":
            assert abs(res.iters - ro.iters) <= tol, (mode, res.iters, ro.iters)
        else:
            assert res.iters <= ro.iters + tol, (mode, res.iters, ro.iters)
        r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, xs.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6
