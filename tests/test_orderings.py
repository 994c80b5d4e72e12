"""Orderings of the cell graph (Sec. 5): RCM, one-way dissection, lines and the
hybrid line-RCM / line-1WD orderings, computed by the library's host code.
CPU tests (no GPU call); one GPU test compares FGMRES iteration counts."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as cg

import abilu_inputs as gen


@pytest.fixture(scope="module")
def ab():
    import __graft_entry__ as g
    g._build_ext().build()
    import paper_1912_00539_gb300 as m
    return m


def _graph(s):
    A = sp.csr_matrix((np.ones(len(s.colind)), s.colind, s.rowptr), shape=(s.n, s.n))
    A = ((A + A.T) > 0).astype(float)
    A.setdiag(0)
    A.eliminate_zeros()
    return A.tocsr()


def _bandwidth(A, perm):
    B = A[perm][:, perm].tocoo()
    return int(np.abs(B.row - B.col).max())


def _is_perm(p, n):
    return np.array_equal(np.sort(p), np.arange(n))


def test_rcm_is_a_permutation_with_scipy_like_bandwidth(ab):
    s = gen.make_system(48, 40, 1, 2, 3, 100.0, order="natural")
    perm, line_of = ab.order(s.rowptr, s.colind, "rcm")
    assert _is_perm(perm, s.n) and np.all(line_of == -1)
    A = _graph(s)
    ref = cg.reverse_cuthill_mckee(A, symmetric_mode=True)
    assert _bandwidth(A, perm) <= 1.1 * _bandwidth(A, ref)
    assert _bandwidth(A, perm) < _bandwidth(A, np.arange(s.n))


def test_rcm_handles_several_components(ab):
    # two disjoint 2x2-block paths and an isolated cell
    rowptr = np.array([0, 2, 4, 6, 8, 9], np.int32)
    colind = np.array([0, 1, 0, 1, 2, 3, 2, 3, 4], np.int32)
    perm, _ = ab.order(rowptr, colind, "rcm")
    assert _is_perm(perm, 5)


def test_one_way_dissection_separators(ab):
    """Removing the cells numbered last (the separators) splits the graph into
    blocks that are contiguous ranges of the new numbering, and no block is
    adjacent to another block."""
    s = gen.make_system(60, 60, 4, 5, 6, 100.0, order="natural")
    perm, _ = ab.order(s.rowptr, s.colind, "1wd")
    assert _is_perm(perm, s.n)
    A = _graph(s)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(s.n)
    P = A[perm][:, perm].tocsr()
    # the separators are the longest suffix of the numbering whose removal
    # leaves the most components (one per block; separator cells put back one
    # by one first attach to a block, so shorter suffixes can tie)
    best = (1, s.n)
    for k in range(s.n - 1, int(0.8 * s.n), -1):
        ncomp, _ = cg.connected_components(P[:k][:, :k], directed=False)
        if ncomp >= best[0]:
            best = (ncomp, k)
    ncomp, k = best
    assert ncomp >= 3 and s.n - k < 0.2 * s.n
    _, lab = cg.connected_components(P[:k][:, :k], directed=False)
    # each block is a contiguous range
    for c in range(ncomp):
        idx = np.flatnonzero(lab == c)
        assert idx.max() - idx.min() + 1 == len(idx)


def _viscous(nx, ny):
    return gen.make_system(nx, ny, 7, 8, 9, 1e4, order="natural", wall_normal_scale=100.0)


def test_lines_follow_the_wall_normal_columns(ab):
    """On the viscous-like grid (wall-normal coupling x100) the lines found
    from the block norms are the grid's wall-normal columns of 2 ny cells."""
    nx, ny = 12, 9
    s = _viscous(nx, ny)
    perm, line_of = ab.order(s.rowptr, s.colind, "line", vals=s.vals, line_threshold=10.0)
    assert _is_perm(perm, s.n)
    assert line_of.max() + 1 == nx and np.all(line_of >= 0)
    cols = gen.line_order(nx, ny)          # new -> natural, column by column
    col_of = np.empty(s.n, np.int64)
    col_of[cols] = np.arange(s.n) // (2 * ny)
    for k in range(nx):
        cells = np.flatnonzero(line_of == k)
        assert len(cells) == 2 * ny and len(set(col_of[cells])) == 1
    # every line is contiguous in the new numbering
    pos = np.empty(s.n, np.int64)
    pos[perm] = np.arange(s.n)
    for k in range(nx):
        p = np.sort(pos[line_of == k])
        assert p[-1] - p[0] + 1 == len(p)


def test_isotropic_grid_has_no_lines(ab):
    s = gen.make_system(20, 20, 1, 2, 3, 100.0, order="natural")
    perm, line_of = ab.order(s.rowptr, s.colind, "line", vals=s.vals, line_threshold=10.0)
    assert np.all(line_of == -1) and np.array_equal(perm, np.arange(s.n))


@pytest.mark.parametrize("kind", ["line-rcm", "line-1wd"])
def test_hybrid_orderings_keep_lines_contiguous(ab, kind):
    nx, ny = 16, 6
    s = _viscous(nx, ny)
    w = np.ones(len(s.colind))             # geometric weights: 1, wall-normal 20
    cols = gen.line_order(nx, ny)
    col_of = np.empty(s.n, np.int64)
    col_of[cols] = np.arange(s.n) // (2 * ny)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    w[(col_of[rows] == col_of[s.colind]) & (rows != s.colind)] = 20.0
    perm, line_of = ab.order(s.rowptr, s.colind, kind, weights=w, line_threshold=5.0)
    assert _is_perm(perm, s.n) and line_of.max() + 1 == nx
    pos = np.empty(s.n, np.int64)
    pos[perm] = np.arange(s.n)
    for k in range(nx):
        p = np.sort(pos[line_of == k])
        assert p[-1] - p[0] + 1 == len(p)


def test_permute_pattern_matches_dense_permutation(ab):
    s = gen.random_pattern_system(60, 150, seed=3)
    rng = np.random.default_rng(1)
    perm = rng.permutation(s.n).astype(np.int32)
    ro, co, src = ab.permute_pattern(s.rowptr, s.colind, perm)
    from oracle import dense
    D = dense.to_blocks(s.rowptr, s.colind, s.vals)
    Dp = dense.to_blocks(ro, co, s.vals[src])
    np.testing.assert_array_equal(Dp, D[perm][:, perm])
    for i in range(s.n):
        c = co[ro[i]:ro[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


def test_order_rejects_bad_input(ab):
    s = gen.small_system(3, 3, seed=1)
    with pytest.raises(ab.AbiluError):
        ab.order(s.rowptr, s.colind, "line")             # no weights or values
    bad = s.colind.copy()
    bad[0] = s.n
    with pytest.raises(ab.AbiluError):
        ab.order(s.rowptr, bad, "rcm")
    with pytest.raises(ab.AbiluError):
        ab.permute_pattern(s.rowptr, s.colind, np.zeros(s.n, np.int32))


@pytest.mark.gpu
def test_line_orderings_help_the_viscous_grid(ab):
    """Viscous-like grid: FGMRES with ABILU needs no more iterations under the
    detected line orderings than under RCM (Sec. 5.1: an ILU on a line
    ordering factors the strongly coupled line blocks exactly)."""
    import torch
    s = _viscous(128, 32)
    iters = {}
    for kind in ("rcm", "line", "line-rcm", "line-1wd", "1wd"):
        perm, _ = ab.order(s.rowptr, s.colind, kind, vals=s.vals, line_threshold=10.0)
        ro, co, src = ab.permute_pattern(s.rowptr, s.colind, perm)
        rp, ci = torch.from_numpy(ro).cuda(), torch.from_numpy(co).cuda()
        A0 = torch.from_numpy(s.vals).cuda()
        A = torch.empty_like(A0)
        ab.gather_blocks(torch.from_numpy(src).cuda(), A0, A)
        b = torch.from_numpy(np.ascontiguousarray(s.b[perm])).cuda()
        pat = ab.Pattern(rp, ci)
        fac = ab.Factors(pat, "f32")
        x = torch.zeros_like(b)
        res = ab.fgmres_solve(pat, A, fac, b, x, restart=50, rtol=1e-6, build_sweeps=8,
                              apply_sweeps_lower=6, apply_sweeps_upper=6, mode="sync")
        assert res.converged, (kind, res)
        iters[kind] = res.iters
    assert iters["line"] <= iters["rcm"], iters
    assert iters["line-rcm"] <= iters["rcm"], iters
    assert iters["line-1wd"] <= iters["rcm"], iters


# ------------------------------------------------- bit-exact against the oracle
# abilu_order is integer work (with comparisons of FP64 coupling weights), so
# it must equal the oracle's orderings (oracle/orderings.c, written from the
# same stated rules) exactly: every permutation entry and every line index.

def _components_system():
    """Several components, isolated cells, and couplings scaled x100 on a
    random subset of edges (lines appear)."""
    rng = np.random.default_rng(21)
    n = 400
    e = rng.integers(0, n, size=(420, 2))
    e = np.unique(np.sort(e[e[:, 0] != e[:, 1]], axis=1), axis=0)
    off = rng.standard_normal((len(e), 2, 4, 4)) * 0.5
    off[rng.random(len(e)) < 0.3] *= 100.0
    rowptr, colind, vals = gen.assemble(n, e, off, 10.0, np.arange(n))
    return gen.System("components", rowptr, colind, vals, np.zeros((n, 4)), np.arange(n), 10.0)


PARITY_GRAPHS = {
    "viscous_1024x256": lambda: gen.make_system(1024, 256, 301, 302, 303, 1e4, order="natural",
                                                wall_normal_scale=100.0),
    "viscous_128x32": lambda: _viscous(128, 32),
    "isotropic_64x64": lambda: gen.make_system(64, 64, 101, 102, 103, 100.0, order="natural"),
    "random_triangles": lambda: gen.random_pattern_system(300, 200, seed=9),
    "components": _components_system,
}
KINDS = ["rcm", "1wd", "line", "line-rcm", "line-1wd"]


@pytest.fixture(scope="module", params=list(PARITY_GRAPHS))
def parity_graph(request):
    return PARITY_GRAPHS[request.param]()


@pytest.mark.parametrize("kind", KINDS)
def test_order_equals_oracle(ab, parity_graph, kind):
    import oracle
    s = parity_graph
    p, l = ab.order(s.rowptr, s.colind, kind, vals=s.vals, line_threshold=10.0)
    po, lo = oracle.order(s.rowptr, s.colind, kind, vals=s.vals, threshold=10.0)
    assert np.array_equal(p, po) and np.array_equal(l, lo)


@pytest.mark.parametrize("kind", ["line", "line-rcm", "line-1wd"])
def test_order_with_caller_weights_equals_oracle(ab, kind):
    """Caller-given (geometric-like) weights: heavy-tailed random per block."""
    import oracle
    s = _components_system()
    w = np.exp(np.random.default_rng(5).normal(0.0, 2.0, len(s.colind)))
    p, l = ab.order(s.rowptr, s.colind, kind, weights=w, line_threshold=6.0)
    po, lo = oracle.order(s.rowptr, s.colind, kind, weights=w, threshold=6.0)
    assert np.array_equal(p, po) and np.array_equal(l, lo)
    assert (l >= 0).sum() > 20


def test_order_matches_hand_worked_cases(ab):
    import test_oracle_orderings as g
    for case in g.golden_cases():
        rp, ci, w = g.golden_pattern(case)
        for kind, perm in g.golden_expectations(case):
            p, line_of = ab.order(rp, ci, kind, weights=w,
                                  line_threshold=case.get("threshold", 10.0))
            assert p.tolist() == perm, (case["name"], kind)
            if "line_of" in case:
                assert line_of.tolist() == case["line_of"], case["name"]
