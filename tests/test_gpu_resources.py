"""Handles give back what they allocate: creating and destroying patterns,
factors, multigrid hierarchies, threshold factorisations and batches many
times leaves the device's free memory where it was (the library allocates
outside the caller's allocator, so this is read from the driver)."""
import gc

import numpy as np
import pytest

import abilu_inputs as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1912_00539_gb300 as m
    return m


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    gc.collect()
    return torch.cuda.mem_get_info()[0]


def test_handles_release_their_memory(ab):
    import torch
    s = gen.workload("inviscid_64x64")
    rp = torch.from_numpy(s.rowptr).cuda()
    ci = torch.from_numpy(s.colind).cuda()
    A = torch.from_numpy(np.ascontiguousarray(s.vals)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(s.b)).cuda()
    x = torch.zeros_like(b)

    def cycle():
        pat = ab.Pattern(rp, ci)
        fac = ab.Factors(pat, "f32")
        ab.fgmres_solve(pat, A, fac, b, x, build_sweeps=2, mode="async")
        mg = ab.Multigrid(pat, A, min_coarse=64)
        ab.fgmres_solve_mg(mg, A, b, x)
        fp, ff = ab.parilut(pat, A, fill=1.5, iters=2, sweeps=1, dtype="f32")
        ab.fgmres_solve(pat, A, ff, b, x, build=False)
        batch = ab.Batch([(rp, ci), (rp, ci)], dtype="f32")
        batch.set_system(0, A, b)
        batch.set_system(1, A, b)
        batch.solve(build_sweeps=2)
        del batch, ff, fp, mg, fac, pat

    cycle()   # first use: lazy module loading, caches
    before = _free_bytes()
    for _ in range(10):
        cycle()
    after = _free_bytes()
    # a leak of any one handle per cycle would be >= several MB x 10 cycles
    assert before - after < 16 * 2 ** 20, (before - after) / 2 ** 20
