"""Spectral-cell discretisation, assembly and DOF partition (oracle, test infrastructure).

Follows the paper's Sec. "Spatial discretization" and Sec. "Partitioning":

  M_ij = int alpha rho N_i N_j,  K_ij = int alpha rho c^2 grad N_i . grad N_j,
  f_i  = int alpha f N_i                                   (Eqs. Mglobal, K, f)

with alpha = 1 in the physical domain and alpha_f in the fictitious domain (the
alpha-scaling of the density, so alpha enters M, K and f alike).  Quadrature
(same section, last paragraph):
  * uncut cells: mass by GLL quadrature on the GLL nodes (diagonal, "nodal
    lumping"); stiffness and load by Gauss-Legendre with p+1 points per axis;
  * cut cells: a spacetree (binary/quad/oct-tree) refined towards the boundary,
    with p+1 GL points per axis on every leaf, for mass, stiffness and load.
Cells with fill ratio below 1e-10 are empty and discarded (2D example).

Partition (Eq. MStructure): I_c = DOFs of any cut cell, I_d = the remaining
active DOFs; M^dd is then diagonal and M^dc = 0.

Readings (see the design notes): spacetree root = level 0, a subcell is
bisected along every axis iff a hole boundary meets its interior, until level
`depth`; every leaf, at any level, gets (p+1)^d GL points.

Global node numbering is the canonical full-grid order: node (i_x, i_y[, i_z])
of the (n_x p + 1) x (n_y p + 1) [x (n_z p + 1)] lattice, x fastest.
Local node order inside a cell is the same (x fastest).

Pins: tests/test_oracle_discretize.py — K symmetric with the constant vector
in its null space, 1^T M 1 equal to the alpha-weighted quadrature volume,
the single-cell eigenfrequency table of Fig. fillRatioHZ, the cell-wise
critical time step of Table criticaltimestepsizes, the analytic standing mode,
the load vector against closed-form integrals and against 1^T M u, the
empty-cell threshold on a 1D cell resolved to 6e-11, K scaling with c^2.
tests/test_oracle_mutations.py checks that mistakes planted here fail them.
"""
import itertools
import numpy as np
import scipy.sparse as sp

from . import basis
from .geometry import UNCUT, CUT, EMPTY, Holes

EMPTY_FILL = 1e-10


class Grid:
    """Cartesian cell grid of the embedding box Omega."""

    def __init__(self, lo, hi, ncells, p):
        self.dim = len(ncells)
        self.lo = np.asarray(lo, dtype=np.float64)[: self.dim]
        self.hi = np.asarray(hi, dtype=np.float64)[: self.dim]
        self.ncells = tuple(int(n) for n in ncells)
        self.p = int(p)
        self.h = (self.hi - self.lo) / np.asarray(self.ncells, dtype=np.float64)
        self.nnodes_axis = tuple(n * self.p + 1 for n in self.ncells)
        self.nnodes = int(np.prod(self.nnodes_axis))
        self.ncell_total = int(np.prod(self.ncells))

    def cell_index(self, ci):
        """Flat cell id (x fastest) of multi-index ci."""
        idx, stride = 0, 1
        for k in range(self.dim):
            idx += ci[k] * stride
            stride *= self.ncells[k]
        return idx

    def cells(self):
        """All cell multi-indices in flat order (x fastest)."""
        rng = [range(n) for n in self.ncells]
        for ci in itertools.product(*reversed(rng)):
            yield tuple(reversed(ci))

    def cell_box(self, ci):
        lo = self.lo + np.asarray(ci) * self.h
        return lo, lo + self.h

    def cell_nodes(self, ci):
        """Global node ids of the (p+1)^d nodes of cell ci, local order x fastest."""
        P = self.p + 1
        ids = np.zeros(P ** self.dim, dtype=np.int64)
        for loc, li in enumerate(itertools.product(*[range(P)] * self.dim)):
            li = tuple(reversed(li))           # li[0] fastest
            g, stride = 0, 1
            for k in range(self.dim):
                g += (ci[k] * self.p + li[k]) * stride
                stride *= self.nnodes_axis[k]
            ids[loc] = g
        return ids

    def node_coords(self):
        """Coordinates of all grid nodes, (nnodes, dim), canonical order."""
        x1, _ = basis.gll_points(self.p)
        axes = []
        for k in range(self.dim):
            c = np.empty(self.nnodes_axis[k])
            for e in range(self.ncells[k]):
                c[e * self.p:(e + 1) * self.p + 1] = self.lo[k] + self.h[k] * (e + (x1 + 1.0) / 2.0)
            axes.append(c)
        mesh = np.meshgrid(*reversed(axes), indexing="ij")
        return np.stack([m.ravel() for m in reversed(mesh)], axis=1)


def tensor_points(x1, w1, dim):
    """Tensor-product rule on [-1,1]^dim from a 1D rule; point order x fastest."""
    pts, wts = [], []
    for idx in itertools.product(*[range(len(x1))] * dim):
        idx = tuple(reversed(idx))
        pts.append([x1[i] for i in idx])
        wts.append(np.prod([w1[i] for i in idx]))
    return np.asarray(pts), np.asarray(wts)


def spacetree_points(geom, box_lo, box_hi, depth, p, dim):
    """GL points of the spacetree leaves of one cut cell.

    Returns reference coordinates in [-1,1]^dim, reference weights (summing to
    2^dim) and the physical mask.  A subcell at level < depth that the boundary
    cuts is bisected in every axis; every leaf gets (p+1)^dim GL points.
    """
    xg, wg = basis.gauss_points(p + 1)
    ref_pts, ref_w = tensor_points(xg, wg, dim)
    h = box_hi - box_lo
    out_x, out_w = [], []

    def visit(rlo, rhi, level):
        plo = box_lo + (rlo + 1.0) / 2.0 * h
        phi = box_lo + (rhi + 1.0) / 2.0 * h
        if level < depth and geom.classify_box(plo, phi) == CUT:
            mid = (rlo + rhi) / 2.0
            for child in itertools.product((0, 1), repeat=dim):
                clo = np.where(np.asarray(child) == 0, rlo, mid)
                chi = np.where(np.asarray(child) == 0, mid, rhi)
                visit(clo, chi, level + 1)
            return
        half = (rhi - rlo) / 2.0
        out_x.append(rlo + (ref_pts + 1.0) * half)
        out_w.append(ref_w * np.prod(half))

    visit(-np.ones(dim), np.ones(dim), 0)
    xr = np.concatenate(out_x)
    wr = np.concatenate(out_w)
    xphys = box_lo + (xr + 1.0) / 2.0 * h
    return xr, wr, geom.physical(xphys)


def shape_functions(p, xr, h):
    """Values N (nq, P^d) and physical gradients G (dim, nq, P^d) of the tensor basis."""
    nodes, _ = basis.gll_points(p)
    dim = xr.shape[1]
    P = p + 1
    vals = [basis.lagrange(nodes, xr[:, k]) for k in range(dim)]
    ders = [basis.lagrange_deriv(nodes, xr[:, k]) * (2.0 / h[k]) for k in range(dim)]
    nq = len(xr)
    N = np.ones((nq, P ** dim))
    G = np.ones((dim, nq, P ** dim))
    for loc, li in enumerate(itertools.product(*[range(P)] * dim)):
        li = tuple(reversed(li))
        for k in range(dim):
            N[:, loc] *= vals[k][:, li[k]]
            for g in range(dim):
                G[g, :, loc] *= (ders[k] if g == k else vals[k])[:, li[k]]
    return N, G


def element_from_points(p, h, xr, wr, alpha_q, rho, c, fvals, reverse=False):
    """K_e, M_e, f_e from quadrature points (Eqs. Mglobal, K, f restricted to one cell).

    reverse: sum over the points in reverse order (the same integral, other
    roundoff; the parity tests use it to sample the rounding spread of the
    assembled system)."""
    if reverse:
        xr, wr, alpha_q = xr[::-1], wr[::-1], np.asarray(alpha_q)[::-1]
        fvals = None if fvals is None else np.asarray(fvals)[::-1]
    N, G = shape_functions(p, xr, h)
    jac = np.prod(h / 2.0)
    wq = wr * jac * alpha_q
    Ke = np.zeros((N.shape[1], N.shape[1]))
    for g in range(G.shape[0]):
        Ke += (G[g] * (wq * rho * c * c)[:, None]).T @ G[g]
    Me = (N * (wq * rho)[:, None]).T @ N
    fe = N.T @ (wq * fvals) if fvals is not None else np.zeros(N.shape[1])
    return Ke, Me, fe


def uncut_element(p, h, rho, c, box_lo, fx, reverse=False):
    """Uncut cell: GL stiffness and load, GLL (diagonal) mass."""
    dim = len(h)
    xg, wg = basis.gauss_points(p + 1)
    xr, wr = tensor_points(xg, wg, dim)
    fv = fx(box_lo + (xr + 1.0) / 2.0 * h) if fx is not None else None
    Ke, _, fe = element_from_points(p, h, xr, wr, np.ones(len(xr)), rho, c, fv, reverse)
    xl, wl = basis.gll_points(p)
    xr2, wr2 = tensor_points(xl, wl, dim)
    _, Me, _ = element_from_points(p, h, xr2, wr2, np.ones(len(xr2)), rho, c, None, reverse)
    return Ke, Me, fe


class Discretization:
    """Assembled SCM system: K, M (CSR, canonical numbering), f_x, partition."""


def all_cell_nodes(grid):
    """Global node ids of every cell, shape (ncells, P^d), cells in flat order,
    local nodes x fastest (same numbering as Grid.cell_nodes)."""
    P, dim = grid.p + 1, grid.dim
    cells = np.array(list(grid.cells()), dtype=np.int64)            # (nc, dim)
    local = np.array([tuple(reversed(li)) for li in itertools.product(*[range(P)] * dim)],
                     dtype=np.int64)                                 # (P^d, dim), x fastest
    ids = np.zeros((len(cells), len(local)), dtype=np.int64)
    stride = 1
    for k in range(dim):
        ids += (cells[:, k:k + 1] * grid.p + local[None, :, k]) * stride
        stride *= grid.nnodes_axis[k]
    return cells, ids


def discretize(grid, geom, alpha, depth, rho=1.0, c0=1.0, cell_c=None, fx=None, quad_reverse=False):
    """Build the assembled system for all non-empty cells of `grid`.

    geom: object with physical(x) and classify_box(lo, hi) (Holes / HalfSpace).
    cell_c: optional per-cell wave speed (flat cell order), default c0 everywhere.
    fx: callable, spatial load f_x(x) for points (n, dim), or None.
    quad_reverse: every element's quadrature summed in reverse point order
    (the same system up to roundoff, about 1e-15 of max |K|).

    Uncut cells all share one reference element: their K_e (c^2-scaled) and
    GLL mass are computed once, and their loads f_e = sum_q w_q |J| f(x_q) N(x_q)
    are evaluated for all uncut cells at once with the same reference values N.
    Cut cells are integrated one by one on their spacetree.
    """
    dim, p = grid.dim, grid.p
    cells, nodes = all_cell_nodes(grid)
    ncell = len(cells)
    ctype = np.zeros(ncell, dtype=np.int8)
    for cid in range(ncell):
        lo, hi = grid.cell_box(cells[cid])
        ctype[cid] = geom.classify_box(lo, hi)
    fill = np.where(ctype == UNCUT, 1.0, 0.0)
    speed = np.full(ncell, float(c0)) if cell_c is None else np.asarray(cell_c, dtype=np.float64)
    jac = np.prod(grid.h / 2.0)
    Pd = (p + 1) ** dim
    rows, cols, kv, mv = [], [], [], []
    fglob = np.zeros(grid.nnodes)

    # Uncut cells: one reference element, scaled by c_e^2 for the stiffness.
    uncut = np.flatnonzero(ctype == UNCUT)
    if len(uncut):
        Ke1, Me1, _ = uncut_element(p, grid.h, rho, 1.0, np.zeros(dim), None, quad_reverse)
        xg, wg = basis.gauss_points(p + 1)
        xr, wr = tensor_points(xg, wg, dim)
        Nq, _ = shape_functions(p, xr, grid.h)                   # (P^d points, P^d basis)
        ids = nodes[uncut]
        rr = np.repeat(ids, Pd, axis=1)
        cc = np.tile(ids, (1, Pd))
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        kv.append((speed[uncut, None] ** 2 * Ke1.ravel()[None, :]).ravel())
        mv.append(np.tile(Me1.ravel(), len(uncut)))
        if fx is not None:
            lo = grid.lo + cells[uncut] * grid.h                     # (n, dim)
            xq = lo[:, None, :] + (xr[None, :, :] + 1.0) / 2.0 * grid.h
            fv = fx(xq.reshape(-1, dim)).reshape(len(uncut), -1)     # (n, points)
            fe = (fv * (wr * jac)[None, :]) @ Nq                     # (n, P^d)
            np.add.at(fglob, ids.ravel(), fe.ravel())

    # Cut cells: spacetree quadrature, one at a time.
    for cid in np.flatnonzero(ctype == CUT):
        lo, hi = grid.cell_box(cells[cid])
        xr, wr, phys = spacetree_points(geom, lo, hi, depth, p, dim)
        eta = float(wr[phys].sum() / wr.sum())
        fill[cid] = eta
        if eta < EMPTY_FILL:
            ctype[cid] = EMPTY
            continue
        aq = np.where(phys, 1.0, alpha)
        fv = fx(lo + (xr + 1.0) / 2.0 * grid.h) if fx is not None else None
        Ke, Me, fe = element_from_points(p, grid.h, xr, wr, aq, rho, float(speed[cid]), fv, quad_reverse)
        ids = nodes[cid]
        rr, cc = np.meshgrid(ids, ids, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        kv.append(Ke.ravel())
        mv.append(Me.ravel())
        np.add.at(fglob, ids, fe)

    n = grid.nnodes
    if rows:
        r = np.concatenate(rows)
        c_ = np.concatenate(cols)
        K = sp.csr_matrix((np.concatenate(kv), (r, c_)), shape=(n, n))
        M = sp.csr_matrix((np.concatenate(mv), (r, c_)), shape=(n, n))
    else:
        K = sp.csr_matrix((n, n))
        M = sp.csr_matrix((n, n))
    K.eliminate_zeros()
    M.eliminate_zeros()

    active = np.zeros(n, dtype=bool)
    is_c = np.zeros(n, dtype=bool)
    active[nodes[ctype != EMPTY].ravel()] = True
    is_c[nodes[ctype == CUT].ravel()] = True
    d = Discretization()
    d.grid, d.K, d.M, d.fx = grid, K, M, fglob
    d.active, d.is_c = active, is_c
    d.is_d = active & ~is_c
    d.cell_type, d.fill = ctype, fill
    d.alpha, d.rho, d.c0, d.cell_c, d.depth = alpha, rho, c0, cell_c, depth
    return d


def uncut_critical_dt(p, h, rho=1.0, c=1.0):
    """Cell-wise critical time step of an uncut cell: 2 / sqrt(lambda_max(K_e, M_e))
    for one free (Neumann) cell (Sec. Motivation eqs.; Table criticaltimestepsizes)."""
    Ke, Me, _ = uncut_element(p, np.asarray(h, dtype=np.float64), rho, c,
                              np.zeros(len(h)), None)
    md = np.diag(Me)
    lam = np.linalg.eigvalsh(Ke / np.sqrt(np.outer(md, md)))
    return 2.0 / np.sqrt(lam.max())
