"""Serving: requests of value updates admitted by HBM footprint, run
concurrently on their own streams; each result is the same alone and in the
mix (bit for bit in synchronous mode, where every request's arithmetic is
independent of the others)."""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


def _requests(n=4, seed=5, arrivals=None, cells=(600, 6000)):
    stream = gen.serving_stream(rate_hz=1000.0, n_requests=n, seed=seed, cells_lo=cells[0],
                                cells_hi=cells[1], n_updates=3)
    from paper_1912_00539_gb300 import serving
    out = []
    for k, r in enumerate(stream):
        t = arrivals[k] if arrivals is not None else 0.0
        out.append(serving.Request(r.rid, t, r.system.rowptr, r.system.colind,
                                   [(v, b) for v, b, _ in r.updates]))
    return out


def test_same_result_alone_and_in_the_mix():
    from paper_1912_00539_gb300 import serving
    reqs = _requests()
    alone = {}
    for r in reqs:
        srv = serving.Server(hbm_budget_bytes=64e9, slots=1, dtype="f32", mode="sync",
                             keep_solutions=True)
        res, _ = srv.run([r])
        alone[r.rid] = res[0]
    srv = serving.Server(hbm_budget_bytes=64e9, slots=4, dtype="f32", mode="sync",
                         keep_solutions=True)
    mix, wall = srv.run(reqs)
    for r, m in zip(reqs, mix):
        a = alone[r.rid]
        assert m.iters == a.iters
        for xa, xm in zip(a.x, m.x):
            np.testing.assert_array_equal(xa, xm)
        for (vals, b), xm in zip(r.updates, m.x):
            res = b - oracle.spmv(r.rowptr, r.colind, vals, xm)
            assert np.linalg.norm(res) / np.linalg.norm(b) <= 1e-6
    # the mix overlapped: some request was admitted before another finished
    iv = sorted((m.admitted, m.finished) for m in mix)
    assert any(iv[k + 1][0] < iv[k][1] for k in range(len(iv) - 1))


def test_async_mix_converges_within_tolerance():
    from paper_1912_00539_gb300 import serving
    reqs = _requests(seed=6)
    srv = serving.Server(hbm_budget_bytes=64e9, slots=4, dtype="f32", mode="async",
                         keep_solutions=True)
    mix, _ = srv.run(reqs)
    for r, m in zip(reqs, mix):
        assert max(m.rel_resid) <= 1e-6
        for (vals, b), xm in zip(r.updates, m.x):
            res = b - oracle.spmv(r.rowptr, r.colind, vals, xm)
            assert np.linalg.norm(res) / np.linalg.norm(b) <= 1e-6


def test_admission_respects_the_memory_budget_and_arrivals():
    from paper_1912_00539_gb300 import serving
    reqs = _requests(n=5, seed=7, arrivals=[0.0, 0.0, 0.05, 0.1, 0.1])
    fps = [serving.footprint_bytes(r.n, r.nnzb, "f32") for r in reqs]
    budget = 2.05 * max(fps)          # at most two requests at a time
    srv = serving.Server(hbm_budget_bytes=budget, slots=8, dtype="f32", mode="sync")
    res, _ = srv.run(reqs)
    for r, m in zip(reqs, res):
        assert m.admitted >= r.arrival - 1e-3
    events = sorted([(m.admitted, 1, fp) for m, fp in zip(res, fps)] +
                    [(m.finished, -1, fp) for m, fp in zip(res, fps)], key=lambda e: (e[0], e[1]))
    used = 0.0
    for _, sgn, fp in events:
        used += sgn * fp
        assert used <= budget + 1e-6
