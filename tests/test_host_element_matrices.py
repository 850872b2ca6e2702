"""Element matrices of the library's host discretisation against the oracle.

The C++ setup integrates every cut cell on its own spacetree (Gauss points on
the leaves, the fictitious part weighted by alpha) and uses one reference form
for uncut cells (Sec. Spatial discretization).  Here its K_e and M_e, read back
through imex_host_element_matrices, are compared entry by entry with the
oracle's (oracle/discretize.py: spacetree_points + element_from_points for cut
cells, uncut_element for uncut ones) on every cut cell and a few uncut and
empty cells of a 2D plate, a small 3D box with a void and a plate with a
wave speed per cell.  The two sum the
same quadrature in different orders, so entries agree to roundoff (1e-12 of
the largest entry of the cell's matrix).  No GPU is needed.
"""
import numpy as np
import pytest

from oracle.discretize import (CUT, EMPTY, EMPTY_FILL, UNCUT, Grid, element_from_points, spacetree_points,
                               uncut_element)
from oracle.geometry import Holes
from paper_2310_14712_gb300 import workloads

TYPE_CODE = {UNCUT: 0, CUT: 1, EMPTY: 2}   # the library's cell-type codes


def _imex():
    from paper_2310_14712_gb300 import imex
    return imex


def _oracle_cell(grid, geom, ci, alpha, depth, rho, c):
    """(type, K_e, M_e) of one cell as the oracle's discretize forms them."""
    lo, hi = grid.cell_box(ci)
    kind = geom.classify_box(lo, hi)
    Pd = (grid.p + 1) ** grid.dim
    if kind == UNCUT:
        Ke, Me, _ = uncut_element(grid.p, grid.h, rho, c, lo, None)
        return UNCUT, Ke, Me
    if kind == CUT:
        xr, wr, phys = spacetree_points(geom, lo, hi, depth, grid.p, grid.dim)
        if wr[phys].sum() / wr.sum() >= EMPTY_FILL:
            aq = np.where(phys, 1.0, alpha)
            Ke, Me, _ = element_from_points(grid.p, grid.h, xr, wr, aq, rho, c, None)
            return CUT, Ke, Me
    return EMPTY, np.zeros((Pd, Pd)), np.zeros((Pd, Pd))


def _check(w, n_uncut=3):
    imex = _imex()
    grid = Grid(w.lo, w.hi, w.ncells, w.p)
    geom = Holes(w.holes, w.dim)
    cells = list(grid.cells())
    kinds = [geom.classify_box(*grid.cell_box(ci)) for ci in cells]
    cut = [k for k, t in enumerate(kinds) if t == CUT]
    uncut = [k for k, t in enumerate(kinds) if t == UNCUT][:n_uncut]
    empty = [k for k, t in enumerate(kinds) if t == EMPTY][:2]
    ids = np.array(cut + uncut + empty, dtype=np.int64)
    assert len(cut) > 0 and len(uncut) > 0
    K, M, types = imex.host_element_matrices(ids, **w.kwargs())
    speed = np.full(len(cells), float(w.c0)) if w.cell_c is None else np.asarray(w.cell_c, dtype=float)
    for q, cid in enumerate(ids):
        kind, Ke, Me = _oracle_cell(grid, geom, cells[cid], w.alpha, w.depth, w.rho, float(speed[cid]))
        assert types[q] == TYPE_CODE[kind], (cid, types[q], kind)
        for lib, ref in ((K[q], Ke), (M[q], Me)):
            scale = max(np.abs(ref).max(), 1e-300)
            assert np.abs(lib - ref).max() <= 1e-12 * scale, (cid, np.abs(lib - ref).max() / scale)
    return types


def test_plate16_cut_and_uncut_cells():
    types = _check(workloads.plate16())
    assert (types == 1).sum() > 10


def test_3d_box_with_a_void():
    w = workloads.Workload("box3d", 3, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (4, 4, 4), 2, 1e-5, 2,
                           np.array([[0.5, 0.45, 0.55, 0.3, 0.25, 0.2]]), np.array([[0.2, 0.3, 0.3]]),
                           3.0, 0.08, 0)
    types = _check(w)
    assert (types == 1).sum() > 5


def test_per_cell_wave_speed():
    # The adjoint's workload: a wave speed per cell in [0.8, 1.2]; cut cells
    # integrate rho c_e^2 on their spacetree, uncut cells scale the reference
    # stiffness by c_e^2 / c0^2 (the mass does not depend on c).
    w = workloads.adjoint()
    assert w.cell_c is not None and np.ptp(w.cell_c) > 0.1
    types = _check(w)
    assert (types == 1).sum() > 10


def test_out_of_range_cell_is_rejected():
    imex = _imex()
    w = workloads.plate16()
    n = int(np.prod(w.ncells))
    with pytest.raises(imex.ImexError):
        imex.host_element_matrices(np.array([n], dtype=np.int64), **w.kwargs())
