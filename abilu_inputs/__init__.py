"""Seeded synthetic inputs shaped like the paper's 2D finite-volume Jacobians.

The paper's test matrices come from a cell-centred finite-volume discretisation
of the compressible Navier-Stokes equations on 2D unstructured grids (Sec. 2):
one 4x4 dense block per pair of face-neighbouring cells, all d+2 = 4 unknowns of
a cell contiguous, and the grid reordered once in preprocessing (Sec. 5).  The
meshes themselves are not available, so this module builds stand-ins:

* a quad grid whose quads are split into two triangles along a seeded random
  diagonal (cells have at most 3 face neighbours, like the paper's triangular /
  hybrid meshes);
* reverse Cuthill-McKee ordering (Sec. 5) and a wall-normal line ordering
  (Sec. 5.1, whole columns as lines);
* block values: off-diagonal blocks N(0,1)*0.5, each directed neighbour pair
  independent (non-symmetric like an upwind Jacobian), the diagonal block a
  diagonal matrix 1/CFL + the absolute row sum of the off-diagonal blocks of that
  block row (a pseudo-time term, Sec. 2);
* right-hand sides N(0,1).

This module is input generation only: it holds none of the preconditioner's or
the solver's arithmetic, and both the CUDA path and the CPU oracle consume the
arrays it produces.  Every array is a plain numpy array; block values are
float64 (nnzb, 4, 4), row-major inside each block.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BS = 4  # unknowns per cell (rho, rho*vx, rho*vy, rho*E), Sec. 2

# edge kinds
EDGE_DIAG = 0        # across the in-quad diagonal
EDGE_VERTICAL = 1    # across a vertical quad edge (tangential direction)
EDGE_HORIZONTAL = 2  # across a horizontal quad edge (wall-normal direction)


@dataclass
class Grid:
    """Triangulated nx x ny quad grid.

    Quad q = j*nx + i is split into cell 2q (the triangle touching the quad's
    bottom edge) and cell 2q+1 (the other one).  ``split[q]`` is True when the
    split runs along '/' (bottom-left to top-right corner).
    """
    nx: int
    ny: int
    split: np.ndarray      # (nx*ny,) bool
    edges: np.ndarray      # (E, 2) int64 natural cell ids, u < v
    kind: np.ndarray       # (E,) int8, EDGE_* codes

    @property
    def ncells(self) -> int:
        return 2 * self.nx * self.ny


def tri_quad_grid(nx: int, ny: int, seed: int) -> Grid:
    """Build the triangulated quad grid; one RNG bit per quad picks the diagonal."""
    if nx < 1 or ny < 1:
        raise ValueError("grid needs nx, ny >= 1")
    rng = np.random.default_rng(seed)
    nq = nx * ny
    split = rng.integers(0, 2, size=nq).astype(bool)
    q = np.arange(nq, dtype=np.int64)
    qi = q % nx
    qj = q // nx
    # in-quad diagonal
    e_diag = np.stack([2 * q, 2 * q + 1], axis=1)
    # vertical quad edge between quad (i,j) and (i+1,j): the right edge of the
    # left quad belongs to its bottom triangle for '/', to its top one for '\';
    # the left edge of the right quad belongs to its top triangle for '/'.
    ql = q[qi < nx - 1]
    qr = ql + 1
    right_owner = np.where(split[ql], 2 * ql, 2 * ql + 1)
    left_owner = np.where(split[qr], 2 * qr + 1, 2 * qr)
    e_vert = np.stack([right_owner, left_owner], axis=1)
    # horizontal quad edge between quad (i,j) and (i,j+1): top triangle of the
    # lower quad, bottom triangle of the upper quad.
    qb = q[qj < ny - 1]
    e_horz = np.stack([2 * qb + 1, 2 * (qb + nx)], axis=1)
    edges = np.concatenate([e_diag, e_vert, e_horz], axis=0)
    kind = np.concatenate([
        np.full(len(e_diag), EDGE_DIAG, np.int8),
        np.full(len(e_vert), EDGE_VERTICAL, np.int8),
        np.full(len(e_horz), EDGE_HORIZONTAL, np.int8),
    ])
    assert np.all(edges[:, 0] < edges[:, 1])
    return Grid(nx, ny, split, edges, kind)


def adjacency(n: int, edges: np.ndarray):
    """Symmetric CSR adjacency (ptr, idx) of an undirected edge list, sorted rows."""
    u = np.concatenate([edges[:, 0], edges[:, 1]])
    v = np.concatenate([edges[:, 1], edges[:, 0]])
    order = np.lexsort((v, u))
    u = u[order]
    v = v[order]
    ptr = np.zeros(n + 1, np.int64)
    np.add.at(ptr, u + 1, 1)
    ptr = np.cumsum(ptr)
    return ptr, v.astype(np.int64)


def _gather_neighbours(ptr, idx, nodes):
    """Concatenated neighbour lists of ``nodes`` and the position of each owner."""
    start = ptr[nodes]
    cnt = ptr[nodes + 1] - start
    owner = np.repeat(np.arange(len(nodes)), cnt)
    offs = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    return idx[np.repeat(start, cnt) + offs], owner


def _bfs_levels(ptr, idx, start, allowed=None):
    n = len(ptr) - 1
    seen = np.zeros(n, bool) if allowed is None else ~allowed.copy()
    seen[start] = True
    levels = [np.array([start], np.int64)]
    while True:
        nb, _ = _gather_neighbours(ptr, idx, levels[-1])
        nb = np.unique(nb[~seen[nb]])
        if len(nb) == 0:
            return levels
        seen[nb] = True
        levels.append(nb)


def pseudo_peripheral_node(ptr, idx, start, allowed=None) -> int:
    """George-Liu pseudo-peripheral node search starting from ``start``."""
    deg = np.diff(ptr)
    r = start
    lv = _bfs_levels(ptr, idx, r, allowed)
    while True:
        last = lv[-1]
        x = int(last[np.lexsort((last, deg[last]))[0]])  # min degree, then min index
        lx = _bfs_levels(ptr, idx, x, allowed)
        if len(lx) > len(lv):
            r, lv = x, lx
        else:
            return r


def rcm_order(ptr, idx) -> np.ndarray:
    """Reverse Cuthill-McKee ordering (Sec. 5).

    Start node: George-Liu pseudo-peripheral node found from the lowest unvisited
    cell of each connected component.  Cuthill-McKee visits the unvisited
    neighbours of each node in queue order sorted by (degree, index); each
    component's order is reversed on its own, components in order of their
    lowest cell.  Returns ``perm`` with perm[new] = old.
    """
    n = len(ptr) - 1
    deg = np.diff(ptr)
    visited = np.zeros(n, bool)
    out = []
    done = 0
    while done < n:
        s0 = int(np.flatnonzero(~visited)[0])
        s = pseudo_peripheral_node(ptr, idx, s0, allowed=~visited)
        comp = [np.array([s], np.int64)]
        visited[s] = True
        frontier = comp[0]
        while len(frontier):
            nb, owner = _gather_neighbours(ptr, idx, frontier)
            keep = ~visited[nb]
            nb, owner = nb[keep], owner[keep]
            if len(nb) == 0:
                break
            o = np.lexsort((nb, deg[nb], owner))
            nb = nb[o]
            _, first = np.unique(nb, return_index=True)
            nxt = nb[np.sort(first)]
            visited[nxt] = True
            comp.append(nxt)
            frontier = nxt
        out.append(np.concatenate(comp)[::-1])
        done += len(out[-1])
    return np.ascontiguousarray(np.concatenate(out))


def line_order(nx: int, ny: int) -> np.ndarray:
    """Wall-normal line ordering (Sec. 5.1): quad columns i = 0..nx-1 in turn,
    inside a column quads by j ascending, bottom triangle then top triangle, so
    every column of cells is a contiguous line.  perm[new] = old."""
    i, j, t = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(2), indexing="ij")
    return (2 * (j * nx + i) + t).reshape(-1).astype(np.int64)


def bandwidth(rowptr, colind) -> int:
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    return int(np.max(np.abs(rows - colind))) if len(colind) else 0


@dataclass
class System:
    """A block sparse system A x = b in block-CSR (BSR) form.

    rowptr int32 (N+1), colind int32 (nnzb) sorted inside each row with the
    diagonal block present in every row, vals float64 (nnzb, 4, 4) row-major
    blocks, b float64 (N, 4).  ``perm[new] = old`` maps the ordering back to
    natural cell ids.
    """
    name: str
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray
    b: np.ndarray
    perm: np.ndarray
    cfl: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.rowptr) - 1

    @property
    def nnzb(self) -> int:
        return len(self.colind)


def offdiag_blocks(grid: Grid, value_seed: int, wall_normal_scale: float = 1.0) -> np.ndarray:
    """(E, 2, 4, 4) off-diagonal blocks; [e, 0] couples u->v (row u, column v),
    [e, 1] couples v->u.  Entries N(0,1)*0.5.  With ``wall_normal_scale`` != 1
    the blocks across horizontal quad edges and across the in-quad diagonal
    (the wall-normal neighbours) are multiplied by it."""
    rng = np.random.default_rng(value_seed)
    off = rng.standard_normal((len(grid.edges), 2, BS, BS)) * 0.5
    if wall_normal_scale != 1.0:
        wn = (grid.kind == EDGE_HORIZONTAL) | (grid.kind == EDGE_DIAG)
        off[wn] *= wall_normal_scale
    return off


@dataclass
class AssemblyPlan:
    """The fixed part of assembling a pattern: the renumbered edge ends and
    the order that sorts the blocks into BSR (rows, then columns)."""
    n: int
    u: np.ndarray
    v: np.ndarray
    order: np.ndarray
    rowptr: np.ndarray
    colind: np.ndarray


def assembly_plan(n: int, edges: np.ndarray, perm: np.ndarray) -> AssemblyPlan:
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    u = inv[edges[:, 0]]
    v = inv[edges[:, 1]]
    rows = np.concatenate([u, v, np.arange(n)])
    cols = np.concatenate([v, u, np.arange(n)])
    o = np.lexsort((cols, rows))
    rows, cols = rows[o], cols[o]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return AssemblyPlan(n, u, v, o, rowptr.astype(np.int32), cols.astype(np.int32))


def assemble_values(plan: AssemblyPlan, off: np.ndarray, cfl: float) -> np.ndarray:
    """Block values of the plan's pattern: the off-diagonal blocks ``off`` and
    diagonal blocks diag(1/CFL + sum over the row's off-diagonal blocks of the
    absolute values in each scalar row)."""
    n = plan.n
    absrow = np.zeros((n, BS))
    np.add.at(absrow, plan.u, np.abs(off[:, 0]).sum(axis=2))
    np.add.at(absrow, plan.v, np.abs(off[:, 1]).sum(axis=2))
    diag = np.zeros((n, BS, BS))
    diag[:, np.arange(BS), np.arange(BS)] = 1.0 / cfl + absrow
    blocks = np.concatenate([off[:, 0], off[:, 1], diag], axis=0)
    return np.ascontiguousarray(blocks[plan.order], dtype=np.float64)


def assemble(n: int, edges: np.ndarray, off: np.ndarray, cfl: float, perm: np.ndarray):
    """BSR arrays in the ordering ``perm`` (perm[new] = old).

    Diagonal block of row i: diag(1/CFL + sum over off-diagonal blocks of row i
    of the absolute values in each scalar row).
    """
    plan = assembly_plan(n, edges, perm)
    return plan.rowptr, plan.colind, assemble_values(plan, off, cfl)


def make_system(nx, ny, grid_seed, value_seed, rhs_seed, cfl, order="rcm",
                wall_normal_scale=1.0, name=None) -> System:
    grid = tri_quad_grid(nx, ny, grid_seed)
    n = grid.ncells
    if order == "rcm":
        ptr, idx = adjacency(n, grid.edges)
        perm = rcm_order(ptr, idx)
    elif order == "line":
        perm = line_order(nx, ny)
    elif order == "natural":
        perm = np.arange(n, dtype=np.int64)
    else:
        raise ValueError(f"unknown ordering {order!r}")
    off = offdiag_blocks(grid, value_seed, wall_normal_scale)
    rowptr, colind, vals = assemble(n, grid.edges, off, cfl, perm)
    b = np.random.default_rng(rhs_seed).standard_normal((n, BS))[perm]
    return System(name or f"tri{nx}x{ny}_{order}", rowptr, colind, vals,
                  np.ascontiguousarray(b), perm, float(cfl),
                  dict(nx=nx, ny=ny, order=order, grid_seed=grid_seed,
                       value_seed=value_seed, rhs_seed=rhs_seed,
                       wall_normal_scale=wall_normal_scale))


# The three single-system workloads.  Sizes: 64x64 quads -> 8,192 cells;
# 512x512 -> 524,288 cells; 1024x256 -> 524,288 cells.
WORKLOADS = {
    "inviscid_64x64": dict(nx=64, ny=64, grid_seed=101, value_seed=102, rhs_seed=103,
                           cfl=100.0, order="rcm"),
    "inviscid_512x512": dict(nx=512, ny=512, grid_seed=201, value_seed=202, rhs_seed=203,
                             cfl=1000.0, order="rcm"),
    "viscous_1024x256_rcm": dict(nx=1024, ny=256, grid_seed=301, value_seed=302,
                                 rhs_seed=303, cfl=1.0e4, order="rcm",
                                 wall_normal_scale=100.0),
    "viscous_1024x256_line": dict(nx=1024, ny=256, grid_seed=301, value_seed=302,
                                  rhs_seed=303, cfl=1.0e4, order="line",
                                  wall_normal_scale=100.0),
}

# solver settings that go with each workload (build sweeps, apply sweeps per
# triangular factor, FGMRES restart, relative tolerance)
SOLVER_SETTINGS = {
    "inviscid_64x64": dict(build_sweeps=4, apply_sweeps=3, restart=30, rtol=1e-6),
    "inviscid_512x512": dict(build_sweeps=6, apply_sweeps=4, restart=30, rtol=1e-6),
    "viscous_1024x256_rcm": dict(build_sweeps=8, apply_sweeps=6, restart=50, rtol=1e-6),
    "viscous_1024x256_line": dict(build_sweeps=8, apply_sweeps=6, restart=50, rtol=1e-6),
}


def workload(name: str) -> System:
    p = dict(WORKLOADS[name])
    return make_system(name=name, **p)


def small_system(nx, ny, seed=0, cfl=100.0, order="rcm", wall_normal_scale=1.0) -> System:
    """Tiny seeded system for tests (three seeds derived from ``seed``)."""
    return make_system(nx, ny, 1000 + 3 * seed, 1001 + 3 * seed, 1002 + 3 * seed, cfl,
                       order=order, wall_normal_scale=wall_normal_scale,
                       name=f"tri{nx}x{ny}_s{seed}")


def _loguniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def batch_specs(n_systems=64, seed=4, cells_lo=2000, cells_hi=200000):
    """Parameters of the uneven batch: cell counts log-uniform in [lo, hi],
    quad aspect ratio nx/ny log-uniform in [1/8, 8], CFL log-uniform in
    [10, 1e4]; one SeedSequence child per system."""
    specs = []
    for k, child in enumerate(np.random.SeedSequence(seed).spawn(n_systems)):
        rng = np.random.default_rng(child)
        cells = _loguniform(rng, cells_lo, cells_hi)
        ar = _loguniform(rng, 1.0 / 8.0, 8.0)
        cfl = _loguniform(rng, 10.0, 1.0e4)
        seeds = rng.integers(0, 2**31 - 1, size=3)
        nq = cells / 2.0
        ny = max(2, int(round(math.sqrt(nq / ar))))
        nx = max(2, int(round(nq / ny)))
        specs.append(dict(nx=nx, ny=ny, grid_seed=int(seeds[0]), value_seed=int(seeds[1]),
                          rhs_seed=int(seeds[2]), cfl=cfl, order="rcm",
                          name=f"batch{k}_{nx}x{ny}"))
    return specs


def batch_systems(n_systems=64, seed=4, cells_lo=2000, cells_hi=200000):
    return [make_system(**s) for s in batch_specs(n_systems, seed, cells_lo, cells_hi)]


@dataclass
class Request:
    """One serving request: a pattern and a sequence of value updates on it."""
    rid: int
    arrival: float            # seconds after the stream starts
    system: System            # pattern + first update
    updates: list             # list of (vals, b) for updates 0..k-1 (update 0 = system)


def value_update(system: System, grid: Grid, base_off: np.ndarray, k: int, cfl0: float,
                 seed: int, plan: AssemblyPlan = None):
    """Values of update k on a fixed pattern: off-diagonal blocks
    base * (1 + 0.1 N(0,1)), CFL_k = CFL_0 * 4^k, diagonal rebuilt."""
    rng = np.random.default_rng(seed)
    off = base_off * (1.0 + 0.1 * rng.standard_normal(base_off.shape))
    cfl = cfl0 * 4.0 ** k
    if plan is None:
        plan = assembly_plan(system.n, grid.edges, system.perm)
    vals = assemble_values(plan, off, cfl)
    b = rng.standard_normal((system.n, BS))[system.perm]
    return vals, np.ascontiguousarray(b), cfl


def serving_stream(rate_hz: float, n_requests: int, seed=5, cells_lo=4000,
                   cells_hi=1_000_000, n_updates=5, cfl0=10.0):
    """Poisson arrivals at ``rate_hz``; sizes log-uniform in [lo, hi] cells;
    each request is ``n_updates`` value updates with CFL ramped x4 per update."""
    ss = np.random.SeedSequence(seed)
    arr_rng = np.random.default_rng(ss.spawn(1)[0])
    gaps = arr_rng.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    out = []
    for rid, child in enumerate(np.random.SeedSequence(seed + 1000).spawn(n_requests)):
        rng = np.random.default_rng(child)
        cells = _loguniform(rng, cells_lo, cells_hi)
        ar = _loguniform(rng, 1.0 / 8.0, 8.0)
        seeds = rng.integers(0, 2**31 - 1, size=3 + n_updates)
        nq = cells / 2.0
        ny = max(2, int(round(math.sqrt(nq / ar))))
        nx = max(2, int(round(nq / ny)))
        grid = tri_quad_grid(nx, ny, int(seeds[0]))
        ptr, idx = adjacency(grid.ncells, grid.edges)
        perm = rcm_order(ptr, idx)
        base = offdiag_blocks(grid, int(seeds[1]))
        plan = assembly_plan(grid.ncells, grid.edges, perm)
        rowptr, colind, vals = plan.rowptr, plan.colind, assemble_values(plan, base, cfl0)
        b = np.random.default_rng(int(seeds[2])).standard_normal((grid.ncells, BS))[perm]
        sysm = System(f"req{rid}_{nx}x{ny}", rowptr, colind, vals, np.ascontiguousarray(b),
                      perm, cfl0, dict(nx=nx, ny=ny))
        ups = [(vals, sysm.b, cfl0)]
        for k in range(1, n_updates):
            ups.append(value_update(sysm, grid, base, k, cfl0, int(seeds[2 + k]), plan))
        out.append(Request(rid, float(arrivals[rid]), sysm, ups))
    return out


@dataclass
class SemilinearCase:
    """A steady model problem r(w) = A w + kappa w|w| - f for the pseudo-time
    continuation driver: `system` carries A (the generator's Jacobian-shaped
    matrix with a small mass term) on its pattern, `w_star` the manufactured
    solution (f = A w* + kappa w*|w*| is formed by whoever evaluates A, not
    here), `shift_scale` s_i = the mean diagonal entry of A_ii (the pseudo-time
    shift of row i is s_i / CFL), `kappa` the nonlinearity."""
    system: System
    w_star: np.ndarray
    shift_scale: np.ndarray
    kappa: float


def semilinear_case(nx, ny, seed=7, kappa=0.5, cfl_base=1.0e4, order="rcm") -> SemilinearCase:
    """Seeded model problem on an nx x ny triangulated quad grid (three grid,
    value and solution seeds derived from ``seed``)."""
    s = make_system(nx, ny, 2000 + 3 * seed, 2001 + 3 * seed, 2002 + 3 * seed, cfl_base,
                    order=order, name=f"semilinear{nx}x{ny}_s{seed}")
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    diag = s.vals[rows == s.colind]                      # [n][4][4], in row order
    scale = np.einsum("nii->n", diag) / BS
    w_star = np.random.default_rng(2003 + 3 * seed).standard_normal((s.n, BS))
    return SemilinearCase(s, np.ascontiguousarray(w_star), np.ascontiguousarray(scale), float(kappa))


def random_pattern_system(n: int, extra_edges: int, seed: int, cfl: float = 10.0,
                          structure: str = "general") -> System:
    """Small system on a random symmetric block pattern (with triangles).

    ``structure``: "general" (symmetric random pattern), "full" (every block
    present), "diagonal" (block diagonal), "lower" / "upper" (the general
    pattern restricted to one triangle plus the diagonal).  Values as in the
    grid systems: off-diagonal N(0,1)*0.5, diagonal 1/CFL + absolute row sum.
    """
    rng = np.random.default_rng(seed)
    if structure == "full":
        iu, ju = np.triu_indices(n, 1)
        edges = np.stack([iu, ju], axis=1).astype(np.int64)
    elif structure == "diagonal":
        edges = np.zeros((0, 2), np.int64)
    else:
        # a path keeps the graph connected, random chords add triangles
        path = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1)
        a = rng.integers(0, n, size=(extra_edges, 2))
        a = a[a[:, 0] != a[:, 1]]
        a = np.sort(a, axis=1)
        edges = np.unique(np.concatenate([path, a]), axis=0).astype(np.int64)
    off = rng.standard_normal((len(edges), 2, BS, BS)) * 0.5
    if structure == "lower":
        off[:, 0] = 0.0          # drop the (u, v) u < v blocks -> only lower
    elif structure == "upper":
        off[:, 1] = 0.0
    rowptr, colind, vals = assemble(n, edges, off, cfl, np.arange(n, dtype=np.int64))
    if structure in ("lower", "upper"):
        # remove the zeroed blocks from the pattern
        rows = np.repeat(np.arange(n), np.diff(rowptr))
        keep = (rows >= colind) if structure == "lower" else (rows <= colind)
        colind, vals = colind[keep], vals[keep]
        rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=n))])
        rowptr = rowptr.astype(np.int32)
    b = rng.standard_normal((n, BS))
    return System(f"rand{n}_{structure}_s{seed}", rowptr, colind, np.ascontiguousarray(vals),
                  b, np.arange(n, dtype=np.int64), float(cfl), dict(structure=structure))
