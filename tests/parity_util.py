"""Shared parity checks of a GPU state against an oracle run (see test_gpu_parity)."""
import numpy as np

from oracle import pipeline
from oracle.geometry import Holes
from oracle.integrators import NewmarkImex


def phys_mask(s, holes):
    return Holes(holes, s.grid.dim).physical(s.grid.node_coords()) & s.disc.active


ORDERINGS = ("NATURAL", "MMD_ATA", "MMD_AT_PLUS_A")
DENSE_INVERSE_MAX = 4000   # implicit DOFs up to which the explicit-inverse variant runs


class _InverseSolve:
    """x = A^{-1} b with the explicitly inverted matrix (a correct FP64 solve
    of another algorithm class than the sparse LU)."""

    def __init__(self, lu, n):
        self.inv = lu.solve(np.eye(n))      # A^{-1}, column by column

    def solve(self, b):
        return self.inv @ b


def ordering_floor(s, ref, nsteps, u0=None, v0=None):
    """Spread of correct answers on the active DOFs: the largest relative L2
    disagreement between the reference run and runs that differ only in how
    the implicit systems are solved: other sparse orderings of the LU and,
    for small implicit partitions, the explicit inverse of the matrices."""
    d = s.disc
    fl = 0.0
    for spec in ORDERINGS:
        alt = NewmarkImex(d.M, d.K, d.fx, s.ft, s.dt, d.is_c, d.is_d, permc_spec=spec)
        fl = max(fl, pipeline.relative_l2(alt.run(nsteps, u0=u0, v0=v0).u, ref.u, d.active))
    nc = int(np.count_nonzero(d.is_c))
    if 0 < nc <= DENSE_INVERSE_MAX:
        alt = NewmarkImex(d.M, d.K, d.fx, s.ft, s.dt, d.is_c, d.is_d)
        alt.S_lu = _InverseSolve(alt.S_lu, nc)
        alt.Mcc_lu = _InverseSolve(alt.Mcc_lu, nc)
        fl = max(fl, pipeline.relative_l2(alt.run(nsteps, u0=u0, v0=v0).u, ref.u, d.active))
    return fl


# Gate on all active DOFs (fictitious nodes included) as a multiple of the
# spread of correct FP64 answers: S = M^cc + dt^2/4 K^cc is ill-conditioned
# (alpha = 1e-5), so fictitious-node values depend on how the implicit systems
# are solved; the device solve composes inverted diagonal blocks with an
# explicitly inverted dense top, two inverse-based stages where each variant
# in the spread uses one method.
FLOOR_FACTOR = 30.0


def check_state(s, ref, st, holes, alpha, nsteps, use_floor=True):
    """Relative L2 gates: physical DOFs <= 1e-11, all active <= max(1e-11,
    FLOOR_FACTOR x floor), CDM history and c-partition velocity/acceleration."""
    act = s.disc.active
    phys = phys_mask(s, holes)
    e_phys = pipeline.relative_l2(st["u"], ref.u, phys)
    e_all = pipeline.relative_l2(st["u"], ref.u, act)
    tol_all = 1e-11
    if use_floor and s.disc.is_c.any() and alpha < 1.0:
        tol_all = max(1e-11, FLOOR_FACTOR * ordering_floor(s, ref, nsteps))
    assert e_phys <= 1e-11, (e_phys, e_all)
    assert e_all <= tol_all, (e_all, tol_all)
    if s.disc.is_d.any():
        assert pipeline.relative_l2(st["u_prev_d"], ref.u_prev_d, s.disc.is_d) <= max(tol_all, 1e-11)
    cphys = phys & s.disc.is_c
    if cphys.any():
        assert pipeline.relative_l2(st["v_c"], ref.v_c, cphys) <= 1e-10
        assert pipeline.relative_l2(st["a_c"], ref.a_c, cphys) <= 1e-10
    return e_phys, e_all
