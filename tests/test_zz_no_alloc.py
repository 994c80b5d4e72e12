"""abilu_apply_noalloc: the allocation-free preconditioner application.

Some callers cannot call cudaMalloc (allocator hooks, pre-reserved memory
pools, graph construction); this entry point serves them from a fixed device
array inside the library.  Its output must equal abilu_apply's (synchronous,
FP64 factors) within the FP64 apply tolerance of the other GPU tests (1e-12),
on two calls in a row (the array keeps the previous call's contents).  This
file is collected last so that a failing run has already run every other test.
"""
import numpy as np
import pytest

import abilu_inputs as gen

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("which", ["grid37x11", "random_triangles", "inviscid_64x64"])
def test_noalloc_apply_matches_apply(which):
    import torch
    import paper_1912_00539_gb300.abilu as ab
    s = {"grid37x11": lambda: gen.small_system(37, 11, seed=2),
         "random_triangles": lambda: gen.random_pattern_system(150, 400, seed=4),
         "inviscid_64x64": lambda: gen.workload("inviscid_64x64")}[which]()
    rowptr = torch.from_numpy(s.rowptr).cuda()
    colind = torch.from_numpy(s.colind).cuda()
    A = torch.from_numpy(s.vals).cuda()
    pat = ab.Pattern(rowptr, colind)
    fac = ab.Factors(pat, "f64")
    fac.build(A, 3, mode="sync")
    X, D = fac.export()
    rng = np.random.default_rng(5)
    for nl, nu in ((3, 3), (4, 2), (1, 1)):
        for call in range(2):  # two calls in a row share the scratch array
            r = torch.from_numpy(rng.standard_normal((s.n, 4))).cuda()
            z_ref = torch.empty_like(r)
            z = torch.full_like(r, np.nan)
            fac.apply(r, z_ref, nl, nu, mode="sync")
            ab.apply_noalloc(rowptr, colind, X, D, r, z, nl, nu)
            torch.cuda.synchronize()
            assert _rel(z.cpu().numpy(), z_ref.cpu().numpy()) < 1e-12, (nl, nu, call)


def test_noalloc_matches_oracle():
    """The same application as the oracle's synchronous FP64 apply on the same
    exported factors (1e-12, the FP64 apply tolerance of the parity tests)."""
    import torch
    import oracle
    import paper_1912_00539_gb300.abilu as ab
    s = gen.random_pattern_system(150, 400, seed=4)
    rowptr = torch.from_numpy(s.rowptr).cuda()
    colind = torch.from_numpy(s.colind).cuda()
    pat = ab.Pattern(rowptr, colind)
    fac = ab.Factors(pat, "f64")
    fac.build(torch.from_numpy(s.vals).cuda(), 2, mode="sync")
    X, D = fac.export()
    Xh, Dh = X.cpu().numpy(), D.cpu().numpy()
    r = np.random.default_rng(9).standard_normal((s.n, 4))
    for nl, nu in ((3, 3), (2, 5)):
        z = torch.empty((s.n, 4), dtype=torch.float64, device="cuda")
        ab.apply_noalloc(rowptr, colind, X, D, torch.from_numpy(r).cuda(), z, nl, nu)
        z_or = oracle.apply(s.rowptr, s.colind, Xh, Dh, r, nl, nu)
        assert _rel(z.cpu().numpy(), z_or) < 1e-12, (nl, nu)


def test_noalloc_rejects_unaligned_views():
    """A view 8 bytes off a 16-byte boundary is refused on the host with
    ABILU_EINVAL (nothing is launched)."""
    import torch
    import paper_1912_00539_gb300.abilu as ab
    s = gen.small_system(4, 3, seed=1)
    n = s.n
    rowptr = torch.from_numpy(s.rowptr).cuda()
    colind = torch.from_numpy(s.colind).cuda()
    X = torch.zeros((s.nnzb, 4, 4), dtype=torch.float64, device="cuda")
    D = torch.zeros((n, 4, 4), dtype=torch.float64, device="cuda")
    buf = torch.zeros(4 * n + 2, dtype=torch.float64, device="cuda")
    r_off = buf[1:1 + 4 * n]          # 8-byte offset, contiguous
    r = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    z = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    Xbuf = torch.zeros(16 * s.nnzb + 2, dtype=torch.float64, device="cuda")
    for args in ((X, D, r_off, z), (X, D, r, buf[1:1 + 4 * n]), (Xbuf[1:1 + 16 * s.nnzb], D, r, z)):
        with pytest.raises(ab.AbiluError) as e:
            ab.apply_noalloc(rowptr, colind, *args, 2, 2)
        assert e.value.status == ab.EINVAL and "aligned" in str(e.value)


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    import paper_1912_00539_gb300.abilu as ab
    n = ab.NOALLOC_MAX_CELLS + 1
    rowptr = torch.arange(n + 1, dtype=torch.int32, device="cuda")
    colind = torch.arange(n, dtype=torch.int32, device="cuda")
    X = torch.zeros((n, 4, 4), dtype=torch.float64, device="cuda")
    D = torch.zeros_like(X)
    r = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(ab.AbiluError) as e:
        ab.apply_noalloc(rowptr, colind, X, D, r, z, 2, 2)
    assert e.value.status == ab.EINVAL and "scratch limit" in str(e.value)
