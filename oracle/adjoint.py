"""Discrete adjoint of the Newmark IMEX time stepping and the gradient of a
receiver misfit with respect to the per-cell wave speed (oracle, test
infrastructure: imported only by the tests, the smoke check and the bench's
CPU leg).

The paper names full-waveform inversion as the application of the method;
this module is the CPU definition of the gradient that such an inversion
needs, for the discrete method of Fig. TrapCDMIMEX exactly (the adjoint of
the discrete step, not a discretised continuous adjoint).

Forward step n -> n+1 (state u_n, u^d_{n-1}, v^c_n, a^c_n; beta = 1/4,
gamma = 1/2):
  1. u^d_{n+1} = 2 u^d_n - u^d_{n-1} + dt^2 (M^dd)^{-1} (f_t(t_n) f^d - K^d u_n)
  2. u^c_p = u^c_n + dt v^c_n + (1/2 - beta) dt^2 a^c_n,  v^c_p = v^c_n + (1 - gamma) dt a^c_n
  3. w = [u^d_{n+1}; u^c_p]
  4. a^c_{n+1} = S^{-1} (f_t(t_{n+1}) f^c - K^c w),  S = M^cc + beta dt^2 K^cc
  5. u^c_{n+1} = u^c_p + beta dt^2 a^c_{n+1},  v^c_{n+1} = v^c_p + gamma dt a^c_{n+1}
Misfit J = 1/2 sum_{n=1..N} sum_r (u_n[x_r] - d_{n,r})^2.

Reverse mode through 5..1 (K, M, S symmetric), with adjoint variables
written with a bar:
  5: ubar^c_p += ubar^c_{n+1};  abar += beta dt^2 ubar^c_{n+1} + gamma dt vbar^c_{n+1};
     vbar^c_p += vbar^c_{n+1}
  4: g = S^{-1} abar;  wbar = -K[:, I_c] g   (d and c rows)
  3: ubar^d_{n+1} += wbar^d;  ubar^c_p += wbar^c
  2: ubar^c_n += ubar^c_p;  vbar^c_n += dt ubar^c_p + vbar^c_p;
     abar^c_n += (1/2 - beta) dt^2 ubar^c_p + (1 - gamma) dt vbar^c_p
  1: h = dt^2 (M^dd)^{-1} ubar^d_{n+1};  ubar_n += -K[:, I_d] h;
     ubar^d_n += 2 ubar^d_{n+1};  ubar^d_{n-1} += -ubar^d_{n+1}
and the misfit adds (u_n - d_n) at the receivers to ubar_n.  With K = sum_e
c_e^2 K_e^(1) (K_e^(1) the element stiffness at unit speed), dK/dc_e =
2 c_e K_e^(1) and dS/dc_e = beta dt^2 dK^cc/dc_e, so step n contributes
  dJ/dc_e += -h^T (dK/dc_e) u_n - g^T (dK/dc_e)[I_c, :] (w + beta dt^2 [0; a^c_{n+1}]).
The initial state (u_0 = v_0 = 0 here) does not depend on c except through
a^c_0 = (M^cc)^{-1}(f_t(0) f^c - K^c u_0), which is independent of c when
u_0 = 0; and the start value u^d_{-1} = u^d_0 - dt v^d_0 + dt^2/2 a^d_0 with
a^d_0 = (M^dd)^{-1}(f_t(0) f^d - K^d u_0), again independent of c for u_0 = 0.

Pins (tests/test_oracle_adjoint.py): the gradient against central finite
differences of J on small problems (with and without cut cells), and J
written out from the forward states.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretize import (UNCUT, CUT, all_cell_nodes, uncut_element, spacetree_points, element_from_points)
from .integrators import BETA, GAMMA

__all__ = ["cell_stiffness_unit", "misfit_and_gradient", "forward_misfit"]


def cell_stiffness_unit(s):
    """Per non-empty cell: (node ids, K_e at unit wave speed)."""
    d = s.disc
    grid = d.grid
    cells, nodes = all_cell_nodes(grid)
    out = {}
    Ke1, _, _ = uncut_element(grid.p, grid.h, d.rho, 1.0, np.zeros(grid.dim), None)
    for cid in range(len(cells)):
        t = d.cell_type[cid]
        if t == UNCUT:
            out[cid] = (nodes[cid], Ke1)
        elif t == CUT:
            lo, hi = grid.cell_box(cells[cid])
            xr, wr, phys = spacetree_points(s.geom, lo, hi, d.depth, grid.p, grid.dim)
            aq = np.where(phys, 1.0, d.alpha)
            Ke, _, _ = element_from_points(grid.p, grid.h, xr, wr, aq, d.rho, 1.0, None)
            out[cid] = (nodes[cid], Ke)
    return out


def _forward(s, nsteps, record):
    """Forward run; record(n, state, w, a_next) is called for n = 0..nsteps-1
    with the state before step n, the vector w of step 4 and a^c_{n+1}."""
    im = s.imex
    st = im.initial_state()
    states = [st]
    for n in range(nsteps):
        Ic = im.Ic
        dt = im.dt
        nxt = im.step(st)
        w = nxt.u.copy()
        w[Ic] = st.u[Ic] + dt * st.v_c[Ic] + (0.5 - BETA) * dt * dt * st.a_c[Ic]
        record(n, st, w, nxt.a_c[Ic].copy())
        st = nxt
        states.append(st)
    return states


def forward_misfit(s, nsteps, rec, data):
    """J = 1/2 sum_{n=1..N} sum_r (u_n[rec_r] - data[n-1, r])^2."""
    st = s.imex.initial_state()
    J = 0.0
    for n in range(nsteps):
        st = s.imex.step(st)
        e = st.u[rec] - data[n]
        J += 0.5 * float(e @ e)
    return J


def misfit_and_gradient(s, cell_c, nsteps, rec, data):
    """J and dJ/dc_e for every cell (zero for empty cells), by the discrete
    adjoint.  s: a setup built with wave speeds cell_c; rec: receiver node
    ids; data: (nsteps, len(rec)) observed traces."""
    im = s.imex
    n_all = im.n
    Id, Ic = im.Id, im.Ic
    dt = im.dt
    K = sp.csr_matrix(s.disc.K)
    KId = K[:, Id]
    KIc = K[:, Ic]
    mdd = im.mdd
    Sfac = getattr(im, "S_lu", None)   # absent when I_c is empty
    hist = []
    _forward(s, nsteps, lambda n, st, w, a1: hist.append((st.u.copy(), w, a1)))
    # Misfit from the recorded states (u_{n+1} is hist[n+1][0]; the last one is recomputed).
    last = im.run(nsteps).u
    us = [h[0] for h in hist[1:]] + [last]
    J = 0.0
    for n in range(nsteps):
        e = us[n][rec] - data[n]
        J += 0.5 * float(e @ e)
    cells = cell_stiffness_unit(s)
    grad = np.zeros(len(cell_c))
    # Adjoint state (of u_{n+1}, u^d_n as "previous", v^c_{n+1}, a^c_{n+1}).
    ubar = np.zeros(n_all)
    ubar_prev_d = np.zeros(n_all)
    vbar = np.zeros(n_all)
    abar = np.zeros(n_all)
    for n in range(nsteps - 1, -1, -1):
        u_n, w, a1 = hist[n]
        # misfit at u_{n+1}
        ubar[rec] += us[n][rec] - data[n]
        # step 5 reverse
        ubar_cp = ubar[Ic].copy()
        abar_c = abar[Ic] + BETA * dt * dt * ubar[Ic] + GAMMA * dt * vbar[Ic]
        vbar_cp = vbar[Ic].copy()
        # step 4 reverse
        g = Sfac.solve(abar_c) if len(Ic) else np.zeros(0)
        wbar = -(KIc @ g)
        # step 3 reverse
        ubar_d_next = ubar[Id] + wbar[Id]
        ubar_cp = ubar_cp + wbar[Ic]
        # step 1 reverse; the state after step n carries u^d_n as its
        # "previous" value, whose adjoint (ubar_prev_d) flows back to u^d_n.
        h = dt * dt * ubar_d_next / mdd
        ubar_n = -(KId @ h)
        ubar_n[Id] += 2.0 * ubar_d_next + ubar_prev_d[Id]
        new_prev_d = np.zeros(n_all)
        new_prev_d[Id] = -ubar_d_next
        # step 2 reverse
        ubar_n[Ic] += ubar_cp
        vbar_n = np.zeros(n_all)
        abar_n = np.zeros(n_all)
        vbar_n[Ic] = dt * ubar_cp + vbar_cp
        abar_n[Ic] = (0.5 - BETA) * dt * dt * ubar_cp + (1.0 - GAMMA) * dt * vbar_cp
        # gradient of step n
        hfull = np.zeros(n_all)
        hfull[Id] = h
        gfull = np.zeros(n_all)
        gfull[Ic] = g
        w2 = w.copy()
        w2[Ic] += BETA * dt * dt * a1
        for cid, (ids, Ke1) in cells.items():
            dK = 2.0 * cell_c[cid] * Ke1
            grad[cid] -= hfull[ids] @ (dK @ u_n[ids]) + gfull[ids] @ (dK @ w2[ids])
        ubar, ubar_prev_d, vbar, abar = ubar_n, new_prev_d, vbar_n, abar_n
    return J, grad
