"""The bounded device-side waits and their timeout status.

The ordered asynchronous build (few chunks per warp) waits on a per-chunk count
of completed sweeps; the staged triangular sweeps wait on their mbarriers.
Each wait gives up after `spin_limit` polls (fgmres_opts), counts a timeout in
the handle's error word, and the call that reads the status returns
ABILU_ETIMEOUT.  The timeout is made on the host: abilu_factors_inject_stall
starts the chunk flags one sweep behind, a value no warp publishes, so every
first wait runs out.  No GPU fault, trap or hang is involved, and the next
solve on the same handle runs normally.
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
    import paper_1912_00539_gb300.abilu as m
    return m


def _dev(s):
    import torch
    return (torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda(),
            torch.from_numpy(s.vals).cuda(), torch.from_numpy(s.b).cuda())


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_stalled_wait_times_out_then_recovers(ab, dtype):
    import torch
    s = gen.small_system(8, 6, seed=3)
    rp, ci, A, b = _dev(s)
    pat = ab.Pattern(rp, ci)
    fac = ab.Factors(pat, dtype)
    x = torch.zeros_like(b)
    fac.inject_stall(True)
    with pytest.raises(ab.AbiluError) as e:
        ab.fgmres_solve(pat, A, fac, b, x, build_sweeps=4, apply_sweeps_lower=3,
                        apply_sweeps_upper=3, mode="async", spin_limit=1000)
    assert e.value.status == ab.ETIMEOUT, str(e.value)
    # the next solve on the same handle, default limit: converges as usual
    x.zero_()
    res = ab.fgmres_solve(pat, A, fac, b, x, build_sweeps=4, apply_sweeps_lower=3,
                          apply_sweeps_upper=3, mode="async")
    assert res.converged and res.rel_resid_true <= 1e-6
    xn = x.cpu().numpy()
    r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, xn)
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(s.b)


def test_stalled_build_reports_through_factors_status(ab):
    """abilu_build alone: the status call after it returns ABILU_ETIMEOUT once,
    then OK (the error word is reset)."""
    s = gen.small_system(8, 6, seed=3)
    rp, ci, A, _ = _dev(s)
    pat = ab.Pattern(rp, ci)
    fac = ab.Factors(pat, "f32")
    fac.set_spin_limit(1000)
    fac.inject_stall(True)
    fac.build(A, 3, mode="async")
    with pytest.raises(ab.AbiluError) as e:
        fac.singular_blocks()
    assert e.value.status == ab.ETIMEOUT
    fac.build(A, 3, mode="async")
    assert fac.singular_blocks() == 0
    with pytest.raises(ab.AbiluError) as e:
        fac.set_spin_limit(-1)
    assert e.value.status == ab.EINVAL


def test_spin_limit_must_be_non_negative(ab):
    import torch
    s = gen.small_system(4, 3, seed=1)
    rp, ci, A, b = _dev(s)
    pat = ab.Pattern(rp, ci)
    fac = ab.Factors(pat, "f32")
    with pytest.raises(ab.AbiluError) as e:
        ab.fgmres_solve(pat, A, fac, b, torch.zeros_like(b), spin_limit=-1)
    assert e.value.status == ab.EINVAL


def test_small_spin_limit_without_stall_still_converges(ab):
    """A small but sufficient limit changes nothing when no wait stalls: the
    synchronous path has no waits and the staged sweeps' barrier waits end
    within a few polls once their copies land (limit 2^16)."""
    import torch
    s = gen.small_system(37, 11, seed=2)
    rp, ci, A, b = _dev(s)
    pat = ab.Pattern(rp, ci)
    fac = ab.Factors(pat, "f32")
    x = torch.zeros_like(b)
    res = ab.fgmres_solve(pat, A, fac, b, x, build_sweeps=4, apply_sweeps_lower=3,
                          apply_sweeps_upper=3, mode="sync", spin_limit=1 << 16)
    assert res.converged and res.rel_resid_true <= 1e-6
