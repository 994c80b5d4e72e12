"""Synthetic input generator: grid topology, orderings, value recipe."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as cg

import abilu_inputs as gen


@pytest.mark.parametrize("nx,ny,E", [(64, 64, 12160), (512, 512, 785408), (1024, 256, 785152)])
def test_edge_counts(nx, ny, E):
    g = gen.tri_quad_grid(nx, ny, 1)
    assert len(g.edges) == E == nx * ny + nx * (ny - 1) + (nx - 1) * ny
    deg = np.bincount(g.edges.reshape(-1), minlength=g.ncells)
    assert deg.max() == 3


def test_grid_has_no_triangles_and_is_connected():
    g = gen.tri_quad_grid(20, 13, 5)
    n = g.ncells
    A = sp.coo_matrix((np.ones(len(g.edges)), (g.edges[:, 0], g.edges[:, 1])), shape=(n, n))
    A = (A + A.T).tocsr()
    assert (A @ A).multiply(A).nnz == 0          # no 3-cycles
    ncomp, _ = cg.connected_components(A)
    assert ncomp == 1


def test_rcm_is_permutation_and_comparable_to_scipy():
    g = gen.tri_quad_grid(64, 64, 101)
    ptr, idx = gen.adjacency(g.ncells, g.edges)
    perm = gen.rcm_order(ptr, idx)
    assert np.array_equal(np.sort(perm), np.arange(g.ncells))
    A = sp.csr_matrix((np.ones(len(idx)), idx, ptr), shape=(g.ncells,) * 2)
    ps = cg.reverse_cuthill_mckee(A, symmetric_mode=True)

    def bw(p):
        B = A[p][:, p].tocoo()
        return np.abs(B.row - B.col).max()
    nat = np.abs(A.tocoo().row - A.tocoo().col).max()
    assert bw(perm) <= 1.1 * bw(ps) and bw(perm) < nat


def test_line_order_makes_columns_contiguous():
    nx, ny = 7, 5
    perm = gen.line_order(nx, ny)
    assert np.array_equal(np.sort(perm), np.arange(2 * nx * ny))
    g = gen.tri_quad_grid(nx, ny, 3)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    # consecutive cells inside a line are neighbours
    es = {(min(a, b), max(a, b)) for a, b in inv[g.edges]}
    for c in range(nx):
        for k in range(2 * ny - 1):
            a = c * 2 * ny + k
            assert (a, a + 1) in es


def test_values_recipe():
    s = gen.make_system(6, 5, 1, 2, 3, cfl=50.0)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    diag = rows == s.colind
    off = ~diag
    # diagonal block = diag(1/CFL + absolute off-diagonal row sum)
    absrow = np.zeros((s.n, 4))
    np.add.at(absrow, rows[off], np.abs(s.vals[off]).sum(axis=2))
    D = s.vals[diag]
    assert np.allclose(D, np.einsum("ij,nj->nij", np.eye(4), absrow + 1 / 50.0), rtol=1e-14)
    # each row sorted and with its diagonal
    for i in range(s.n):
        c = s.colind[s.rowptr[i]:s.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c
    assert abs(np.std(s.vals[off]) - 0.5) < 0.1


def test_orderings_are_the_same_matrix():
    a = gen.make_system(8, 6, 1, 2, 3, 100.0, order="rcm")
    b = gen.make_system(8, 6, 1, 2, 3, 100.0, order="line")
    from oracle import dense
    Da = dense.to_blocks(a.rowptr, a.colind, a.vals)
    Db = dense.to_blocks(b.rowptr, b.colind, b.vals)
    ia = np.empty_like(a.perm)
    ia[a.perm] = np.arange(a.n)
    ib = np.empty_like(b.perm)
    ib[b.perm] = np.arange(b.n)
    # natural ordering of both must coincide
    np.testing.assert_array_equal(Da[ia][:, ia], Db[ib][:, ib])
    np.testing.assert_array_equal(a.b[ia], b.b[ib])


def test_batch_specs_ranges():
    specs = gen.batch_specs(64)
    cells = np.array([2 * s["nx"] * s["ny"] for s in specs])
    assert len(specs) == 64 and cells.min() >= 1500 and cells.max() <= 230000
    assert all(10 <= s["cfl"] <= 1e4 for s in specs)


def test_server_arena_sizing():
    """The server's arena bytes grow linearly with its capacity, shrink with
    narrower factors, and the budget sizing picks the largest arena that fits
    (host arithmetic only, no GPU call)."""
    import __graft_entry__ as g
    g._build_ext().build()              # the package loads the CUDA library (no GPU call here)
    import paper_1912_00539_gb300.abilu as ab
    from paper_1912_00539_gb300 import serving
    small = ab.server_arena_bytes(64 * 1000, 4 * 64 * 1000)
    big = ab.server_arena_bytes(64 * 100000, 4 * 64 * 100000)
    assert 95 * small < big < 101 * small
    f64, f32, bf16 = (ab.server_arena_bytes(65536, 262144, dtype=d) for d in ("f64", "f32", "bf16"))
    assert f64 > f32 > bf16
    # the Krylov basis of FGMRES(30), 62 vectors of 32 bytes per cell, dominates
    assert 62 * 32 * 65536 < f32 < 2.5 * 62 * 32 * 65536
    for budget in (3e8, 4e9):
        c = serving.arena_cells_for_budget(budget)
        assert c % 64 == 0
        assert ab.server_arena_bytes(c, int(4.2 * c)) <= budget
        assert ab.server_arena_bytes(c + 64, int(4.2 * (c + 64))) > budget
    assert serving.arena_cells_for_budget(1e3) == 0


def test_autotune_cache_keys():
    from paper_1912_00539_gb300 import autotune
    assert autotune.cfl_bucket(10.0, 1e4) == "cfl1e1-1e4"
    assert autotune.cfl_bucket(12.0, 900.0) == "cfl1e1-1e3"
    k = autotune._key("GB300", "f32", 524288, autotune.cfl_bucket(100.0, 100.0))
    assert k == "GB300|f32|2^19|cfl1e2-1e2"
    assert len({c for _, _, m, c in autotune.DEFAULT_GRID if m == "async"}) == 3
