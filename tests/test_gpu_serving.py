"""Serving by continuous batching (serving.Server over abilu_server_*):
requests of value updates share every step's launches; each result is the
same alone and in the mix (bit for bit in synchronous mode, where a system's
arithmetic does not depend on the others nor on its place in the arena, also
after departures re-lay the arena and move the warm-start factors); memory
stays inside the budget and a departed request's share is reused."""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


def _requests(n=4, seed=5, arrivals=None, cells=(600, 6000), n_updates=(3, 5, 2, 4)):
    stream = gen.serving_stream(rate_hz=1000.0, n_requests=n, seed=seed, cells_lo=cells[0],
                                cells_hi=cells[1], n_updates=max(n_updates))
    from paper_1912_00539_gb300 import serving
    out = []
    for k, r in enumerate(stream):
        t = arrivals[k] if arrivals is not None else 0.0
        nu = n_updates[k % len(n_updates)]
        out.append(serving.Request(r.rid, t, r.system.rowptr, r.system.colind,
                                   [(v, b) for v, b, _ in r.updates[:nu]]))
    return out


def _check_residuals(reqs, res):
    for r, m in zip(reqs, res):
        for (vals, b), xm in zip(r.updates, m.x):
            rr = b - oracle.spmv(r.rowptr, r.colind, vals, xm)
            assert np.linalg.norm(rr) / np.linalg.norm(b) <= 1e-6


def test_same_result_alone_and_in_the_mix():
    from paper_1912_00539_gb300 import serving
    reqs = _requests(n=5, arrivals=[0.0, 0.0, 0.0, 0.0, 0.002])
    alone = {}
    for r in reqs:
        srv = serving.Server(hbm_budget_bytes=2e9, dtype="f32", mode="sync", keep_solutions=True)
        res, _ = srv.run([r])
        alone[r.rid] = res[0]
    for groups in (1, 2):   # one arena, or two stepped on their own threads and streams
        srv = serving.Server(hbm_budget_bytes=2e9, dtype="f32", mode="sync", keep_solutions=True,
                             groups=groups)
        mix, wall = srv.run(reqs)
        for r, m in zip(reqs, mix):
            a = alone[r.rid]
            assert m.iters == a.iters, (groups, r.rid)
            for xa, xm in zip(a.x, m.x):
                np.testing.assert_array_equal(xa, xm)
        _check_residuals(reqs, mix)
        steps = [s for m in mix for s in m.steps]
        if groups == 1:   # the requests shared steps; the arena was laid out again as they left
            assert max(steps) >= 4 and len(set(steps)) >= 3
        else:             # both groups stepped
            assert max(steps) >= 2


def test_async_mix_converges_within_tolerance():
    from paper_1912_00539_gb300 import serving
    reqs = _requests(seed=6)
    srv = serving.Server(hbm_budget_bytes=2e9, dtype="f32", mode="async", keep_solutions=True)
    mix, _ = srv.run(reqs)
    for m in mix:
        assert max(m.rel_resid) <= 1e-6
    _check_residuals(reqs, mix)


@pytest.mark.parametrize("dtype", ["bf16", "f64"])
def test_other_factor_dtypes_alone_and_in_the_mix(dtype):
    from paper_1912_00539_gb300 import serving
    reqs = _requests(n=3, seed=8, n_updates=(2, 3, 2))
    alone = {}
    for r in reqs:
        res, _ = serving.Server(2e9, dtype=dtype, mode="sync", keep_solutions=True).run([r])
        alone[r.rid] = res[0]
    mix, _ = serving.Server(2e9, dtype=dtype, mode="sync", keep_solutions=True).run(reqs)
    for r, m in zip(reqs, mix):
        for xa, xm in zip(alone[r.rid].x, m.x):
            np.testing.assert_array_equal(xa, xm)
    _check_residuals(reqs, mix)


def test_admission_waits_for_room_and_memory_stays_in_the_budget():
    """An arena with room for about two of the requests: a request waits until
    a departure frees room (first come, first served), is never admitted
    before it arrives, and the device memory in use stays within the budget;
    after the stream every request's own memory has been released."""
    import torch
    from paper_1912_00539_gb300 import serving
    reqs = _requests(n=5, seed=7, arrivals=[0.0, 0.0, 0.01, 0.02, 0.02], cells=(3000, 4000),
                     n_updates=(3, 3, 3, 3, 3))
    import paper_1912_00539_gb300.abilu as ab
    padded = sorted((r.n + 63) // 64 * 64 for r in reqs)
    cap = padded[-1] + padded[-2] + 64          # any two requests, never three
    assert sum(padded[:3]) > cap
    budget = (ab.server_arena_bytes(cap, int(4.2 * cap), 64, "f32", 30) + 4096) / 0.9
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    srv = serving.Server(hbm_budget_bytes=budget, dtype="f32", mode="sync", groups=1)
    assert srv.cells == cap
    srv._engine()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    res, _ = srv.run(reqs)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    for r, m in zip(reqs, res):
        assert m.admitted >= r.arrival - 1e-3
    assert max(s for m in res for s in m.steps) <= 2
    slack = 64 << 20   # the CUDA context and torch's own small allocations
    used0 = total - free0
    assert max(u for _, u in srv.memory_samples) <= used0 + budget + slack
    assert abs((total - free2) - (total - free1)) <= slack   # patterns released, arena kept
    assert (total - free1) - used0 <= srv.arena_bytes + slack


def test_step_rejects_a_partial_list():
    import torch
    import paper_1912_00539_gb300.abilu as ab
    s1 = gen.small_system(8, 6, seed=1)
    s2 = gen.small_system(9, 5, seed=2)
    eng = ab.NativeServer(4096, 16384, 4, "f32", 30)
    ids = [eng.add(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
           for s in (s1, s2)]
    A = [torch.from_numpy(s1.vals).cuda()]
    b = [torch.from_numpy(s1.b).cuda()]
    x = [torch.zeros_like(b[0])]
    with pytest.raises(ab.AbiluError) as e:
        eng.step(ids[:1], A, b, x)
    assert e.value.status == ab.EINVAL
    with pytest.raises(ab.AbiluError) as e:   # the Krylov workspace is sized for FGMRES(30)
        eng.step(ids, A + [torch.from_numpy(s2.vals).cuda()],
                 b + [torch.from_numpy(s2.b).cuda()], x + [torch.zeros(s2.n, 4, dtype=torch.float64,
                                                                     device="cuda")], restart=40)
    assert e.value.status == ab.EINVAL
    u = eng.usage()
    assert u["used"]["systems"] == 2 and u["used"]["rows"] == 256   # 96 and 90 cells, 128 rows each
    big = gen.small_system(45, 45, seed=3)      # 4,050 cells: 4,096 rows > 4,096 - 256 free
    assert eng.add(torch.from_numpy(big.rowptr).cuda(), torch.from_numpy(big.colind).cuda()) is None
    pbig = ab.Pattern(torch.from_numpy(big.rowptr).cuda(), torch.from_numpy(big.colind).cuda())
    assert eng.add_pattern(pbig) is None and pbig.handle    # refused: the caller keeps it
    eng.remove(ids[1])                          # room again once a system leaves
    assert eng.usage()["used"]["rows"] == 128
    fits = gen.small_system(40, 40, seed=3)     # 3,200 cells
    pfit = ab.Pattern(torch.from_numpy(fits.rowptr).cuda(), torch.from_numpy(fits.colind).cuda())
    assert eng.add_pattern(pfit) is not None and not pfit.handle   # the server owns it now


@pytest.mark.slow
def test_full_size_requests_alone_and_in_the_mix():
    """Requests of 4k to 1M cells (the serving workload's range, log-uniform)
    with the 5-update CFL ramp, synchronous FP32: each request's solutions are
    bit for bit those it gets alone, every update converges to 1e-6 (checked
    with the oracle's SpMV), and the steps were shared."""
    from paper_1912_00539_gb300 import serving
    stream = gen.serving_stream(rate_hz=1e6, n_requests=5, seed=12, cells_lo=4000,
                                cells_hi=1_000_000, n_updates=5)
    # the range's ends are covered: the smallest and largest of the stream
    # replaced by 4k- and ~1M-cell requests
    big = gen.serving_stream(rate_hz=1e6, n_requests=1, seed=40, cells_lo=900_000,
                             cells_hi=1_000_000, n_updates=5)[0]
    small = gen.serving_stream(rate_hz=1e6, n_requests=1, seed=41, cells_lo=4000,
                               cells_hi=4100, n_updates=5)[0]
    pool = stream[:3] + [big, small]
    reqs = [serving.Request(k, 0.0, r.system.rowptr, r.system.colind,
                            [(v, b) for v, b, _ in r.updates[: (5 if k % 2 == 0 else 3)]])
            for k, r in enumerate(pool)]
    budget = 60e9
    alone = {}
    for r in reqs:
        res, _ = serving.Server(budget, dtype="f32", mode="sync", keep_solutions=True).run([r])
        alone[r.rid] = res[0]
    mix, _ = serving.Server(budget, dtype="f32", mode="sync", keep_solutions=True).run(reqs)
    for r, m in zip(reqs, mix):
        assert m.iters == alone[r.rid].iters
        for xa, xm in zip(alone[r.rid].x, m.x):
            np.testing.assert_array_equal(xa, xm)
    _check_residuals(reqs, mix)
    assert max(r.n for r in reqs) > 850_000 and min(r.n for r in reqs) < 4200
