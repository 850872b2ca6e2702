"""The paper's comparison schemes on the same spectral cell discretisation
(oracle, test infrastructure: imported only by the tests, the smoke check and
the bench's CPU leg).

  * "imex": Newmark IMEX (Fig. TrapCDMIMEX), the method itself.
  * "cdm": central differences on every DOF with the consistent SCM mass
    (Eqs. CDMstep, CDMacc): M is GLL-diagonal on I_d and the consistent cut
    blocks on I_c (Eq. MStructure), so each step is a diagonal update of I_d
    and a solve with M^cc.
  * "cdm_hrz": central differences with every cut-cell mass matrix
    HRZ-lumped (Sec. "Lumping of Cut Cells", Eqs. HRZ): the diagonal of M_e
    scaled by m_e / sum_k M_e,kk, with m_e = 1^T M_e 1 the element mass, and
    the off-diagonal entries dropped.  The assembled mass is diagonal.
  * "trapezoidal": the trapezoidal Newmark method (beta = 1/4, gamma = 1/2,
    Fig. implicitNewmark) on every DOF with the consistent mass.

Critical steps (Table criticaltimestepsizes): cell-wise, 2 / sqrt(lambda_max(K_e,
M_e)) per cell for the mass the scheme uses; for central differences on an
assembled system the global lambda_max is at most the largest element
lambda_max (the element eigenvalue bound), so the smallest cell-wise step is
a stable choice.

Pins (tests/test_oracle_schemes.py): HRZ on a diagonal matrix is the
identity, preserves the element mass, and gives the textbook halves for the
consistent linear bar element; the assembled HRZ mass is diagonal with the
consistent total mass; the element eigenvalue bound against the global
eigenvalue of a small plate for both masses; without cut cells all three
central-difference forms coincide with IMEX, and the trapezoidal scheme
equals IMEX with I_d empty; central differences stay bounded below their
critical step and grow above it.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .discretize import CUT, UNCUT, all_cell_nodes, element_from_points, spacetree_points, uncut_element
from .integrators import NewmarkImex, cdm, trapezoidal_newmark

SCHEMES = ("imex", "cdm", "cdm_hrz", "trapezoidal")


def hrz_lump(Me):
    """HRZ lumping of one element mass matrix (Eqs. HRZ)."""
    Me = np.asarray(Me, dtype=np.float64)
    d = np.diag(Me).copy()
    return np.diag(d * (Me.sum() / d.sum()))


def cell_matrices(s):
    """Per non-empty cell: (node ids, K_e, M_e) at the setup's wave speeds."""
    d = s.disc
    grid = d.grid
    cells, nodes = all_cell_nodes(grid)
    speed = np.full(len(cells), d.c0) if d.cell_c is None else np.asarray(d.cell_c, dtype=np.float64)
    out = {}
    for cid in range(len(cells)):
        t = d.cell_type[cid]
        if t == UNCUT:
            Ke, Me, _ = uncut_element(grid.p, grid.h, d.rho, float(speed[cid]), np.zeros(grid.dim), None)
        elif t == CUT:
            lo, hi = grid.cell_box(cells[cid])
            xr, wr, phys = spacetree_points(s.geom, lo, hi, d.depth, grid.p, grid.dim)
            aq = np.where(phys, 1.0, d.alpha)
            Ke, Me, _ = element_from_points(grid.p, grid.h, xr, wr, aq, d.rho, float(speed[cid]), None)
        else:
            continue
        out[cid] = (nodes[cid], Ke, Me)
    return out


def hrz_mass(s, cells=None):
    """Assembled mass with every cut-cell block HRZ-lumped (diagonal)."""
    d = s.disc
    cells = cell_matrices(s) if cells is None else cells
    diag = np.zeros(d.grid.nnodes)
    for cid, (ids, _, Me) in cells.items():
        Mt = hrz_lump(Me) if d.cell_type[cid] == CUT else Me
        np.add.at(diag, ids, np.diag(Mt))
    return sp.diags(diag).tocsr()


def cellwise_critical_dt(s, mass="consistent", cells=None):
    """(uncut, smallest cut) cell-wise critical steps 2 / sqrt(lambda_max(K_e, M_e))."""
    d = s.disc
    cells = cell_matrices(s) if cells is None else cells
    lam_u, lam_c = 0.0, 0.0
    for cid, (_, Ke, Me) in cells.items():
        Mt = hrz_lump(Me) if (mass == "hrz" and d.cell_type[cid] == CUT) else Me
        lam = sla.eigh(Ke, Mt, eigvals_only=True)[-1]
        if d.cell_type[cid] == CUT:
            lam_c = max(lam_c, lam)
        else:
            lam_u = max(lam_u, lam)
    dt_u = 2.0 / np.sqrt(lam_u) if lam_u > 0 else np.inf
    dt_c = 2.0 / np.sqrt(lam_c) if lam_c > 0 else np.inf
    return dt_u, dt_c


class SchemeState:
    """u_n on every active DOF; u_prev = u_{n-1} (central differences) or None;
    v, a (trapezoidal) or None."""

    def __init__(self, u, u_prev=None, v=None, a=None):
        self.u, self.u_prev, self.v, self.a = u, u_prev, v, a


def run(s, scheme, nsteps, u0=None, v0=None, M_hrz=None, permc_spec="COLAMD"):
    """nsteps of `scheme` from (u0, v0) (default zero) with the setup's dt,
    force and masks; the system is restricted to the active DOFs.  permc_spec:
    column ordering of the sparse LUs (the IMEX scheme uses the setup's own)."""
    d = s.disc
    n = d.grid.nnodes
    act = np.flatnonzero(d.active)
    u0 = np.zeros(n) if u0 is None else np.asarray(u0, dtype=np.float64)
    v0 = np.zeros(n) if v0 is None else np.asarray(v0, dtype=np.float64)
    if scheme == "imex":
        st = s.imex.run(nsteps, u0=u0, v0=v0)
        return SchemeState(st.u, st.u_prev_d)
    K = sp.csr_matrix(d.K)[act][:, act]
    fx = np.asarray(d.fx)[act]
    if scheme == "trapezoidal":
        M = sp.csr_matrix(d.M)[act][:, act]
        u, v, a = trapezoidal_newmark(M, K, fx, s.ft, s.dt, nsteps, u0[act], v0[act], permc_spec=permc_spec)
        out = [np.zeros(n) for _ in range(3)]
        for o, x in zip(out, (u, v, a)):
            o[act] = x
        return SchemeState(out[0], v=out[1], a=out[2])
    if scheme == "cdm":
        M = sp.csr_matrix(d.M)[act][:, act]
    elif scheme == "cdm_hrz":
        M = (hrz_mass(s) if M_hrz is None else M_hrz)[act][:, act]
    else:
        raise ValueError(f"unknown scheme {scheme!r}")
    u, u_prev = cdm(M, K, fx, s.ft, s.dt, nsteps, u0[act], v0[act], permc_spec=permc_spec)
    uf, pf = np.zeros(n), np.zeros(n)
    uf[act], pf[act] = u, u_prev
    return SchemeState(uf, pf)


def imex_all_implicit(s):
    """Newmark IMEX with I_d empty (every active DOF implicit)."""
    d = s.disc
    return NewmarkImex(d.M, d.K, d.fx, s.ft, s.dt, d.active, np.zeros_like(d.active))
