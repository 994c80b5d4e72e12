"""Batched solves: every system of a batch gets the result it gets alone.

The batch runs the build, triangular sweeps and SpMV of all systems in the same
launches over a padded block-diagonal concatenation and keeps a separate
FGMRES state per system.  In synchronous mode each system's arithmetic is the
single-system arithmetic except the order of the dot-product reductions, so
iteration counts must agree and solutions agree to the solve tolerance.
"""
import numpy as np
import pytest

import abilu_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import torch
    assert torch.cuda.is_available()
    import paper_1912_00539_gb300 as m
    return m


def _dev(s):
    import torch
    return (torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda(),
            torch.from_numpy(np.ascontiguousarray(s.vals)).cuda(),
            torch.from_numpy(np.ascontiguousarray(s.b)).cuda())


def _systems():
    return [gen.small_system(5, 4, seed=31),                        # 40 cells (< one 64-row chunk)
            gen.small_system(37, 11, seed=32),                      # 814 cells, ragged
            gen.make_system(30, 20, 41, 42, 43, cfl=10.0),          # easy: converges early
            gen.make_system(40, 40, 44, 45, 46, cfl=1e4),           # harder
            gen.random_pattern_system(150, 400, seed=33),           # pattern with triangles
            gen.workload("inviscid_64x64")]


@pytest.mark.parametrize("dtype,mode", [("f64", "sync"), ("f32", "sync"), ("f32", "async")])
def test_batch_matches_single_solves(ab, dtype, mode):
    import torch
    systems = _systems()
    devs = [_dev(s) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in devs], dtype=dtype)
    c = batch.counts()
    assert c["nsys"] == len(systems) and c["rows"] % 64 == 0
    assert c["rows"] == sum(-(-s.n // 64) * 64 for s in systems)
    for k, d in enumerate(devs):
        batch.set_system(k, d[2], d[3])
    opts = dict(restart=30, rtol=1e-6, build_sweeps=4, apply_sweeps_lower=3,
                apply_sweeps_upper=3, mode=mode)
    res = batch.solve(**opts)
    for k, (s, d) in enumerate(zip(systems, devs)):
        x = torch.empty_like(d[3])
        batch.solution(k, x)
        xn = x.cpu().numpy()
        r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, xn)
        assert res[k].converged and res[k].rel_resid_true <= 1e-6, (k, res[k])
        assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6
        # alone
        pat = ab.Pattern(d[0], d[1])
        fac = ab.Factors(pat, dtype)
        xa = torch.zeros_like(d[3])
        ra = ab.fgmres_solve(pat, d[2], fac, d[3], xa, **opts)
        if mode == "sync":
            assert res[k].iters == ra.iters, (k, res[k].iters, ra.iters)
            scale = np.abs(xa.cpu().numpy()).max()
            assert np.abs(xn - xa.cpu().numpy()).max() <= 1e-6 * scale
        else:
            assert abs(res[k].iters - ra.iters) <= max(2, ra.iters // 5), (k, res[k].iters, ra.iters)


def test_batch_value_update_and_warm_start(ab):
    """New values on the same patterns, factors warm-started (init=previous)."""
    import torch
    systems = _systems()[:3]
    devs = [_dev(s) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in devs], dtype="f32")
    for k, d in enumerate(devs):
        batch.set_system(k, d[2], d[3])
    batch.solve(build_sweeps=3, mode="sync")
    rng = np.random.default_rng(7)
    for k, s in enumerate(systems):
        vals = s.vals * (1.0 + 0.01 * rng.standard_normal(s.vals.shape))
        bnew = rng.standard_normal(s.b.shape)
        batch.set_system(k, torch.from_numpy(vals).cuda(), torch.from_numpy(bnew).cuda())
        systems[k] = gen.System(s.name, s.rowptr, s.colind, vals, bnew, s.perm, s.cfl)
    res = batch.solve(build_sweeps=1, mode="sync", init="previous")
    for k, s in enumerate(systems):
        x = torch.empty((s.n, 4), dtype=torch.float64, device="cuda")
        batch.solution(k, x)
        r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
        assert res[k].converged
        assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6


@pytest.mark.parametrize("rtol", [1e-8, 1e-10])
def test_batch_tight_tolerances_and_the_graph_key(ab, rtol):
    """Tolerances below 1e-7 take the classical Gram-Schmidt step with the
    explicit norm: every system converges to rtol (checked with the oracle's
    SpMV) in the same iterations as its single-system solve (synchronous
    FP64).  The batch first solves at 1e-6 (single-reduction step), so the
    second solve must not replay the first one's captured cycle: the graph
    key holds the tolerance and the Gram-Schmidt form."""
    import torch
    systems = _systems()[:4]
    devs = [_dev(s) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in devs], dtype="f64")
    for k, d in enumerate(devs):
        batch.set_system(k, d[2], d[3])
    base = dict(restart=30, build_sweeps=4, apply_sweeps_lower=3, apply_sweeps_upper=3,
                mode="sync")
    batch.solve(rtol=1e-6, **base)
    res = batch.solve(rtol=rtol, **base)
    for k, (s, d) in enumerate(zip(systems, devs)):
        x = torch.empty_like(d[3])
        batch.solution(k, x)
        r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
        assert res[k].converged and np.linalg.norm(r) / np.linalg.norm(s.b) <= rtol * 1.001, k
        pat = ab.Pattern(d[0], d[1])
        fac = ab.Factors(pat, "f64")
        xa = torch.zeros_like(d[3])
        ra = ab.fgmres_solve(pat, d[2], fac, d[3], xa, rtol=rtol, **base)
        assert res[k].iters == ra.iters, (k, res[k].iters, ra.iters)


@pytest.mark.parametrize("rtol,reorth", [(1e-6, False), (1e-8, False), (1e-8, True)])
def test_batch_steps_wider_than_the_fused_tile(ab, rtol, reorth):
    """Each Arnoldi step of the batch forms w = A z_j in the kernel that takes
    the first three dot products of the first Gram-Schmidt pass (and ||w||^2 in
    the single-reduction form); wider steps re-read the CTA's own entries of w
    for the remaining tiles.  In every Gram-Schmidt form (single reduction at
    1e-6, classical with the explicit norm at 1e-8, CGS2) each system takes
    its single-system iteration count (synchronous FP64) and reaches rtol, and
    at least one system runs steps past the fourth (two past the fused tile)."""
    import torch
    systems = _systems()[:4]
    devs = [_dev(s) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in devs], dtype="f64")
    for k, d in enumerate(devs):
        batch.set_system(k, d[2], d[3])
    opts = dict(restart=30, rtol=rtol, build_sweeps=2, apply_sweeps_lower=1, apply_sweeps_upper=1,
                mode="sync", reorth=reorth)
    res = batch.solve(**opts)
    assert max(r.iters for r in res) > 4
    for k, (s, d) in enumerate(zip(systems, devs)):
        x = torch.empty_like(d[3])
        batch.solution(k, x)
        r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
        assert res[k].converged and np.linalg.norm(r) / np.linalg.norm(s.b) <= rtol * 1.001, k
        pat = ab.Pattern(d[0], d[1])
        fac = ab.Factors(pat, "f64")
        xa = torch.zeros_like(d[3])
        ra = ab.fgmres_solve(pat, d[2], fac, d[3], xa, **opts)
        assert res[k].iters == ra.iters, (k, res[k].iters, ra.iters)


@pytest.mark.parametrize("rtol,reorth", [(1e-6, False), (1e-8, False), (1e-8, True)])
def test_batch_fp64_solutions_equal_the_oracle(ab, rtol, reorth):
    """Every system of an FP64 synchronous batch against the oracle's FGMRES
    (modified Gram-Schmidt) on that system alone: the same iteration count
    and, the iterates being the same in exact arithmetic, solutions that
    differ by rounding only, in every Gram-Schmidt form (single reduction at
    1e-6, classical with the explicit norm at 1e-8, CGS2).  Measured 3.7e-16
    to 3.2e-15 relative (2-norm) over 10-20 iterations; bound 1e-11, as for
    the single-system solve."""
    import torch
    systems = _systems()
    devs = [_dev(s) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in devs], dtype="f64")
    for k, d in enumerate(devs):
        batch.set_system(k, d[2], d[3])
    res = batch.solve(restart=30, rtol=rtol, build_sweeps=2, apply_sweeps_lower=1,
                      apply_sweeps_upper=1, mode="sync", reorth=reorth)
    for k, (s, d) in enumerate(zip(systems, devs)):
        x = torch.empty_like(d[3])
        batch.solution(k, x)
        Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 2)
        xo, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, 1, 1, restart=30,
                               rtol=rtol)
        assert res[k].converged and res[k].iters == ro.iters, (k, res[k].iters, ro.iters)
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-11, k


def test_batch_rejects_bad_input(ab):
    import torch
    s = gen.small_system(3, 3, seed=34)
    rp = torch.from_numpy(s.rowptr).cuda()
    ci = torch.from_numpy(s.colind.copy()).cuda()
    ci[0], ci[1] = int(s.colind[1]), int(s.colind[0])   # unsorted row
    with pytest.raises(ab.AbiluError):
        ab.Batch([(rp, ci)])


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_graph_and_host_driven_cycles_agree(ab, mode, monkeypatch):
    """The replayed cycle graph (conditional steps) and the host-driven loop run
    the same kernels on the same data; in sync mode the results are identical."""
    import torch
    systems = _systems()[:4]
    devs = [_dev(s) for s in systems]
    out = {}
    for graph in (True, False):
        if graph:
            monkeypatch.delenv("ABILU_NO_GRAPH", raising=False)
        else:
            monkeypatch.setenv("ABILU_NO_GRAPH", "1")
        batch = ab.Batch([(d[0], d[1]) for d in devs], dtype="f32")
        for k, d in enumerate(devs):
            batch.set_system(k, d[2], d[3])
        opts = dict(restart=10, rtol=1e-6, build_sweeps=4, apply_sweeps_lower=3,
                    apply_sweeps_upper=3, mode=mode)
        runs = []
        for rep in range(2):                  # second solve replays the captured graph
            l0 = ab.kernel_launches()
            res = batch.solve(**opts)
            torch.cuda.synchronize()
            launches = ab.kernel_launches() - l0
            xs = []
            for k, d in enumerate(devs):
                x = torch.empty_like(d[3])
                batch.solution(k, x)
                xs.append(x.cpu().numpy())
            runs.append((res, xs, launches))
        out[graph] = runs
        del batch
    for graph, runs in out.items():
        for res, xs, launches in runs:
            assert all(r.converged for r in res)
            # at least init + one cycle of every step's kernels
            assert launches >= 10, launches
    if mode == "sync":
        for (rg, xg, _), (rh, xh, _) in zip(out[True], out[False]):
            assert [r.iters for r in rg] == [r.iters for r in rh]
            for a, b in zip(xg, xh):
                np.testing.assert_array_equal(a, b)


@pytest.mark.slow
def test_full_batch_of_64_uneven_systems(ab):
    """The batched workload at full size: 64 systems of 2k-200k cells
    (log-uniform, seeded aspect ratios and CFL 10-1e4) in one batch, FP32
    factors, synchronous 4 build / 3+3 apply sweeps: every system converges to
    a true FP64 residual <= 1e-6 (the oracle's SpMV) with the FP64 oracle's
    iteration count for that system within 10% (at least 1)."""
    import torch
    systems = gen.batch_systems()
    assert len(systems) == 64
    devs = [_dev(s) for s in systems]
    batch = ab.Batch([(d[0], d[1]) for d in devs], dtype="f32")
    for k, d in enumerate(devs):
        batch.set_system(k, d[2], d[3])
    res = batch.solve(restart=30, rtol=1e-6, build_sweeps=4, apply_sweeps_lower=3,
                      apply_sweeps_upper=3, mode="sync")
    for k, (s, d) in enumerate(zip(systems, devs)):
        x = torch.empty_like(d[3])
        batch.solution(k, x)
        r = s.b - oracle.spmv(s.rowptr, s.colind, s.vals, x.cpu().numpy())
        assert res[k].converged and np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-6, k
        Xo, Do, _ = oracle.bilu_sync(s.rowptr, s.colind, s.vals, 4)
        _, ro = oracle.fgmres(s.rowptr, s.colind, s.vals, Xo, Do, s.b, 3, 3, restart=30, rtol=1e-6)
        assert abs(res[k].iters - ro.iters) <= max(1, ro.iters // 10), (k, res[k].iters, ro.iters)


def test_autotuner_picks_a_converging_candidate_and_keeps_its_launch_shape(tmp_path):
    """The batch autotuner over sweep counts, mode and the asynchronous build's
    ticket size: the choice converges, is the fastest of those timed, its
    build chunk stays set on the batch, and the cache keyed by size and CFL
    range returns it without timing again."""
    import torch
    import paper_1912_00539_gb300 as ab
    from paper_1912_00539_gb300 import autotune
    systems = [gen.small_system(30, 20, seed=1, cfl=10.0), gen.small_system(41, 13, seed=2, cfl=1e3)]
    dev = [(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda()) for s in systems]
    batch = ab.Batch(dev, dtype="f32")
    for k, s in enumerate(systems):
        batch.set_system(k, torch.from_numpy(s.vals).cuda(), torch.from_numpy(s.b).cuda())
    grid = [(2, 2, "sync", 0), (4, 3, "async", 64), (4, 3, "async", 256)]
    cache = str(tmp_path / "tune.json")
    cells = sum(s.n for s in systems)
    ch = autotune.tune_batch(batch, cells, cfl_range=(10.0, 1e3), grid=grid, cache_path=cache)
    assert (ch.build_sweeps, ch.apply_sweeps, ch.mode, ch.build_chunk) in grid
    res = batch.solve(build_sweeps=ch.build_sweeps, apply_sweeps_lower=ch.apply_sweeps,
                      apply_sweeps_upper=ch.apply_sweeps, mode=ch.mode)
    assert all(r.converged for r in res)
    again = autotune.tune_batch(batch, cells, cfl_range=(10.0, 1e3), grid=[(6, 4, "sync", 0)],
                                cache_path=cache)
    assert again == ch          # from the cache, not re-timed on the new grid
    other = autotune.tune_batch(batch, cells, cfl_range=(1e3, 1e4), grid=[(6, 4, "sync", 0)],
                                cache_path=cache)
    assert (other.build_sweeps, other.mode) == (6, "sync")   # another CFL range: tuned anew


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-4), ("bf16", 2e-2)])
def test_build_chunk_sizes_give_converging_async_builds(dtype, tol):
    """Every allowed ticket size is a legal asynchronous iteration: the
    factors reach sequential block ILU(0) with enough sweeps, whether a ticket
    is one sub-chunk (32, 64), several 64-block sub-chunks spread over the
    work list (128, 256, 512) or several 32-block ones (96, 160); bad sizes
    are refused."""
    import torch
    import oracle
    import paper_1912_00539_gb300.abilu as ab
    s = gen.small_system(37, 11, seed=2)
    pat = ab.Pattern(torch.from_numpy(s.rowptr).cuda(), torch.from_numpy(s.colind).cuda())
    A = torch.from_numpy(s.vals).cuda()
    Xs, Ds, _ = oracle.bilu0_seq(s.rowptr, s.colind, s.vals)
    fac = ab.Factors(pat, dtype)
    for c in (32, 64, 96, 128, 160, 256, 512):
        fac.set_build_chunk(c)
        fac.build(A, 2 * s.n + 4, mode="async")
        X, D = fac.export()
        X, D = X.cpu().numpy(), D.cpu().numpy()
        assert np.abs(X - Xs).max() / np.abs(Xs).max() < tol, c
        assert np.abs(D - Ds).max() / np.abs(Ds).max() < tol, c
    for bad in (16, 48, 1024):
        with pytest.raises(ab.AbiluError):
            fac.set_build_chunk(bad)
