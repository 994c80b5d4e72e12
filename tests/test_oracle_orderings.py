"""Pins of the oracle's orderings (oracle/orderings.c; Sec. 5, 5.1, 5.2):
small graphs worked by hand from the stated rules (tests/golden/
orderings_worked.json), the input generator's independent numpy RCM, scipy's
RCM bandwidth, and the structural properties that one-way dissection and the
line orderings must have."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as cg

import abilu_inputs as gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "orderings_worked.json")


def golden_cases():
    return json.load(open(GOLDEN))["cases"]


def golden_pattern(case):
    """(rowptr, colind, weights) of a golden case: every cell has its diagonal
    block, each undirected edge both off-diagonal blocks."""
    n = case["n"]
    rows = [{i: 0.0} for i in range(n)]
    for e in case.get("edges", []):
        rows[e[0]][e[1]] = rows[e[1]][e[0]] = 1.0
    for a, b, w in case.get("wedges", []):
        rows[a][b] = rows[b][a] = w
    rp, ci, ws = [0], [], []
    for r in rows:
        for j in sorted(r):
            ci.append(j)
            ws.append(r[j])
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(ws)


def golden_expectations(case):
    """[(kind, perm)] of a golden case."""
    if "kind" in case:
        return [(case["kind"], case["perm"])]
    return list(case["perm"].items())


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_oracle_matches_hand_worked_orderings(case):
    rp, ci, w = golden_pattern(case)
    for kind, perm in golden_expectations(case):
        p, line_of = oracle.order(rp, ci, kind, weights=w, threshold=case.get("threshold", 10.0))
        assert p.tolist() == perm, (kind, p.tolist())
        if "line_of" in case:
            assert line_of.tolist() == case["line_of"]


def _natural(nx, ny, seed, wall=1.0, cfl=100.0):
    return gen.make_system(nx, ny, seed, seed + 1, seed + 2, cfl, order="natural",
                           wall_normal_scale=wall)


@pytest.mark.parametrize("nx,ny,seed", [(64, 64, 101), (128, 32, 7), (1024, 256, 301)])
def test_rcm_equals_the_generators_independent_rcm(nx, ny, seed):
    """abilu_inputs.rcm_order (vectorised numpy, written separately) and the
    oracle give the same permutation."""
    g = gen.tri_quad_grid(nx, ny, seed)
    ptr, idx = gen.adjacency(g.ncells, g.edges)
    s = _natural(nx, ny, seed)
    p, _ = oracle.order(s.rowptr, s.colind, "rcm")
    assert np.array_equal(p, gen.rcm_order(ptr, idx))


def test_rcm_with_components_equals_the_generators():
    """Several components and isolated cells: per-component reversal."""
    rng = np.random.default_rng(11)
    n = 200
    edges = rng.integers(0, n, size=(150, 2))
    edges = edges[edges[:, 0] != edges[:, 1]]
    ptr, idx = gen.adjacency(n, np.unique(np.sort(edges, axis=1), axis=0))
    A = sp.csr_matrix((np.ones(len(idx)), idx, ptr), shape=(n, n)) + sp.eye(n)
    A = A.tocsr()
    A.sort_indices()
    p, _ = oracle.order(A.indptr.astype(np.int32), A.indices.astype(np.int32), "rcm")
    assert np.array_equal(p, gen.rcm_order(ptr, idx))
    assert cg.connected_components(A)[0] > 10


def _graph(s):
    A = sp.csr_matrix((np.ones(len(s.colind)), s.colind, s.rowptr), shape=(s.n, s.n))
    A = ((A + A.T) > 0).astype(float)
    A.setdiag(0)
    A.eliminate_zeros()
    return A.tocsr()


def _bandwidth(A, perm):
    B = A[perm][:, perm].tocoo()
    return int(np.abs(B.row - B.col).max())


@pytest.mark.parametrize("kind", ["rcm", "1wd", "line", "line-rcm", "line-1wd"])
def test_every_kind_is_a_permutation(kind):
    s = _natural(48, 40, 1, wall=100.0)
    p, _ = oracle.order(s.rowptr, s.colind, kind, vals=s.vals)
    assert np.array_equal(np.sort(p), np.arange(s.n))


def test_rcm_bandwidth_against_scipy():
    s = _natural(48, 40, 1)
    p, _ = oracle.order(s.rowptr, s.colind, "rcm")
    A = _graph(s)
    ref = cg.reverse_cuthill_mckee(A, symmetric_mode=True)
    assert _bandwidth(A, p) <= 1.1 * _bandwidth(A, ref)


def test_one_way_dissection_structure():
    """The cells numbered last (the separators) split the rest into blocks
    that are contiguous ranges of the new numbering and never adjacent to
    another block."""
    s = _natural(60, 60, 4)
    p, _ = oracle.order(s.rowptr, s.colind, "1wd")
    P = _graph(s)[p][:, p].tocsr()
    # the separators are the longest suffix whose removal leaves the most
    # components (separator cells put back one by one first attach to a block)
    best = (1, s.n)
    for k in range(s.n - 1, int(0.8 * s.n), -1):
        ncomp, _ = cg.connected_components(P[:k][:, :k], directed=False)
        if ncomp >= best[0]:
            best = (ncomp, k)
    ncomp, k = best
    assert ncomp >= 3 and s.n - k < 0.2 * s.n
    _, lab = cg.connected_components(P[:k][:, :k], directed=False)
    for c in range(ncomp):
        idx = np.flatnonzero(lab == c)
        assert idx.max() - idx.min() + 1 == len(idx)


def test_lines_are_the_wall_normal_columns():
    """On the viscous-like grid (wall-normal couplings x100) the lines found
    from the block norms are exactly the quad columns' cells, each in
    wall-normal order, and the LINE ordering keeps each one contiguous."""
    nx, ny = 32, 16
    s = _natural(nx, ny, 7, wall=100.0, cfl=1e4)
    p, line_of = oracle.order(s.rowptr, s.colind, "line", vals=s.vals)
    assert line_of.min() == 0 and len(set(line_of.tolist())) == nx
    cells = np.arange(s.n)
    column = (cells // 2) % nx
    for l in range(nx):
        members = cells[line_of == l]
        assert len(set(column[members].tolist())) == 1 and len(members) == 2 * ny
    pos = np.empty(s.n, np.int64)
    pos[p] = np.arange(s.n)
    for l in range(nx):
        q = np.sort(pos[line_of == l])
        assert q[-1] - q[0] == len(q) - 1
    # along each line the quad row index never decreases by more than one
    # step between neighbours in the line (wall-normal order)
    row = (cells // 2) // nx
    for l in range(nx):
        order = p[np.sort(pos[line_of == l])]
        assert np.all(np.abs(np.diff(row[order])) <= 1)


def test_no_lines_on_an_isotropic_grid():
    s = _natural(40, 40, 3)
    _, line_of = oracle.order(s.rowptr, s.colind, "line", vals=s.vals)
    assert np.all(line_of == -1)
