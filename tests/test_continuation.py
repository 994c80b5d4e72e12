"""Pseudo-time continuation driver (Sec. 2): the CFL rule of Eq. (cfl) on the
host, and on the GPU a steady model problem marched to its manufactured
solution, every step's matrix assembled on the device and solved by FGMRES +
ABILU with factors warm-started from the previous step."""
import math

import numpy as np
import pytest

import abilu_inputs as gen


def _driver():
    import __graft_entry__ as g
    g._build_ext().build()                  # the package loads the CUDA library (no GPU call)
    from paper_1912_00539_gb300 import continuation
    return continuation


def test_cfl_rule():
    """Eq. (cfl): growth with exponent 0.25 while the residual falls, shrink with
    0.3 when it does not (ratio <= 1), kept between the start and max values."""
    c = _driver()
    assert math.isclose(c.cfl_update(10.0, 4.0, 1.0, 10.0, 1e4), 10.0 * 4.0 ** 0.25)
    assert math.isclose(c.cfl_update(100.0, 1.0, 2.0, 10.0, 1e4), 100.0 * 0.5 ** 0.3)
    assert c.cfl_update(100.0, 1.0, 1.0, 10.0, 1e4) == 100.0          # ratio 1: exponent 0.3, 1^0.3
    assert c.cfl_update(20.0, 1.0, 1e6, 10.0, 1e4) == 10.0            # clamped below
    assert c.cfl_update(9e3, 1e8, 1.0, 10.0, 1e4) == 1e4              # clamped above
    assert c.cfl_update(50.0, 1.0, 0.0, 10.0, 1e4) == 1e4             # converged exactly


def test_semilinear_case_is_consistent():
    case = gen.semilinear_case(9, 7)
    s = case.system
    assert case.w_star.shape == (s.n, 4) and case.shift_scale.shape == (s.n,)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    d = s.vals[rows == s.colind]
    assert np.allclose(case.shift_scale, np.einsum("nii->n", d) / 4)
    assert np.all(case.shift_scale > 0)


def _residual_cpu(case, f, w):
    import oracle
    s = case.system
    return oracle.spmv(s.rowptr, s.colind, s.vals, w) + case.kappa * w * np.abs(w) - f


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,mode", [("f32", "async"), ("f64", "sync")])
def test_continuation_reaches_manufactured_solution(dtype, mode):
    import torch
    import oracle
    import paper_1912_00539_gb300 as ab
    from paper_1912_00539_gb300.continuation import (PseudoTimeSolver, SemilinearProblem,
                                                     cfl_update)
    case = gen.semilinear_case(40, 30)
    s = case.system
    f = oracle.spmv(s.rowptr, s.colind, s.vals, case.w_star) + case.kappa * case.w_star * np.abs(case.w_star)
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    A = torch.from_numpy(s.vals).cuda()
    prob = SemilinearProblem(pat, A, torch.from_numpy(f).cuda(), case.kappa)
    drv = PseudoTimeSolver(pat, prob.residual, prob.jacobian,
                           torch.from_numpy(case.shift_scale).cuda(), dtype=dtype, mode=mode)
    w = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    log = drv.run(w, rel_tol=1e-6, max_steps=300)
    wn = w.cpu().numpy()
    r0 = np.linalg.norm(f[:, 3])
    r = _residual_cpu(case, f, wn)
    # converged in the energy component, checked with an independent residual
    assert np.linalg.norm(r[:, 3]) <= 1.01e-6 * r0, (len(log), log[-1])
    assert np.linalg.norm(wn - case.w_star) <= 1e-4 * np.linalg.norm(case.w_star)
    # the CFL sequence is Eq. (cfl) applied to the logged residual norms
    rn0 = np.linalg.norm(f)
    cfl, prev = 10.0, rn0
    for st in log:
        assert math.isclose(st.cfl, cfl, rel_tol=1e-12), (st.step, st.cfl, cfl)
        cfl, prev = cfl_update(cfl, prev, st.rnorm, 10.0, 1e4), st.rnorm
    assert max(st.cfl for st in log) > 10.0
    # every linear solve reached its 0.1 drop or stopped at the 60-iteration cap
    assert all(st.lin_rel_resid <= 0.1 or st.lin_iters >= 60 for st in log)
