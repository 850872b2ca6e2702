"""Time integrators on an assembled second-order system M u'' + K u = f_t(t) f_x
(oracle, test infrastructure).  Sec. "Time integration".

  * cdm: central differences, two-step "sum step" (Eq. CDMstep) with the
    acceleration from the equation of motion (Eq. CDMacc); M is factorised once
    (diagonal M needs no factorisation).
  * trapezoidal_newmark: predictor / solve with S = M + beta dt^2 K / corrector,
    beta = 1/4, gamma = 1/2 (Eqs. Newmark1, Newmark2; Fig. implicitNewmark).
  * newmark_imex: the Newmark IMEX method of Fig. TrapCDMIMEX: a diagonal CDM
    step on the explicit DOFs I_d, then the Newmark prediction, acceleration
    calculation with S = M^cc + beta dt^2 K^cc, and correction on the implicit
    DOFs I_c, the prediction using the new explicit values u^d_{n+1}.

Readings taken (listed with the design notes):
  * CDM start value (the flowcharts do not give u_{-1}): Taylor start
    u_{-1} = u_0 - dt v_0 + dt^2/2 a_0 with M a_0 = f_t(0) f_x - K u_0.
  * The IMEX initial-acceleration box reads f_x and u_n where the block
    dimensions force f_x^c and u^c_n.
  * t_n = n dt is formed as a product, not accumulated; exactly `nsteps`
    steps are taken (the flowchart's "t_{n+1} <= T" test).
  * Direct solves use scipy.sparse.linalg.splu (SuperLU), as the paper's 2D
    study does.

Pins (tests/test_oracle_integrators.py): the exact discrete single-mode
solutions u_n = cos(n theta) phi with cos(theta) = 1 - lambda dt^2 / 2 (CDM)
and cos(theta) = (1 - lambda dt^2/4) / (1 + lambda dt^2/4) (trapezoidal); the
IMEX special cases I_c = {} (= CDM) and I_d = {} (= trapezoidal); the ten
spring-coupled masses of Sec. "Spring-coupled masses" (critical steps 3.9086e-2 s
and 1.0154 s, second-order convergence to the Helmholtz solution, bounded
energy at 0.99 dt_crit^explicit and growth at 1.01).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BETA = 0.25
GAMMA = 0.5


def _csc(A):
    return sp.csc_matrix(A)


def _is_diagonal(A):
    A = sp.coo_matrix(A)
    return bool(np.all(A.row == A.col) or A.nnz == 0)


def cdm(M, K, fx, ft, dt, nsteps, u0, v0, callback=None, permc_spec="COLAMD"):
    """Central difference method (Eqs. CDMstep, CDMacc). Returns (u_n, u_{n-1}).
    permc_spec: column ordering of the sparse LU of a non-diagonal M."""
    n = M.shape[0]
    if _is_diagonal(M):
        md = np.asarray(M.diagonal())
        solve = lambda b: b / md
    else:
        lu = spla.splu(_csc(M), permc_spec=permc_spec)
        solve = lu.solve
    u = np.array(u0, dtype=np.float64)
    a0 = solve(ft(0.0) * fx - K @ u)
    u_prev = u - dt * np.asarray(v0) + 0.5 * dt * dt * a0
    for k in range(nsteps):
        t = k * dt
        a = solve(ft(t) * fx - K @ u)
        u_next = 2.0 * u - u_prev + dt * dt * a
        u_prev, u = u, u_next
        if callback is not None:
            callback(k + 1, u)
    return u, u_prev


def trapezoidal_newmark(M, K, fx, ft, dt, nsteps, u0, v0, callback=None, permc_spec="COLAMD"):
    """Trapezoidal Newmark, predictor-corrector form (Fig. implicitNewmark).
    Returns (u, v, a).  permc_spec: column ordering of the sparse LUs."""
    u = np.array(u0, dtype=np.float64)
    v = np.array(v0, dtype=np.float64)
    a = spla.splu(_csc(M), permc_spec=permc_spec).solve(ft(0.0) * fx - K @ u)
    S = spla.splu(_csc(M + BETA * dt * dt * K), permc_spec=permc_spec)
    for k in range(nsteps):
        t1 = (k + 1) * dt
        u_pred = u + dt * v + (0.5 - BETA) * dt * dt * a
        v_pred = v + (1.0 - GAMMA) * dt * a
        a = S.solve(ft(t1) * fx - K @ u_pred)
        u = u_pred + BETA * dt * dt * a
        v = v_pred + GAMMA * dt * a
        if callback is not None:
            callback(k + 1, u)
    return u, v, a


class ImexState:
    """State of the Newmark IMEX recurrence after n steps.

    u: full vector u_n (both partitions); u_prev_d: u^d_{n-1} on I_d (zeros
    elsewhere); v_c, a_c: velocity and acceleration on I_c (zeros elsewhere).
    """

    def __init__(self, n, u, u_prev_d, v_c, a_c):
        self.n, self.u, self.u_prev_d, self.v_c, self.a_c = n, u, u_prev_d, v_c, a_c


class NewmarkImex:
    """Newmark IMEX (Fig. TrapCDMIMEX) on an assembled system.

    is_c: boolean mask of the implicit DOFs I_c; is_d: mask of the explicit DOFs
    I_d (default: complement of is_c).  DOFs in neither set are inactive and
    stay zero.  M restricted to I_d must be diagonal with no coupling to I_c
    (Eq. MStructure).
    """

    def __init__(self, M, K, fx, ft, dt, is_c, is_d=None, permc_spec="COLAMD"):
        M = sp.csr_matrix(M)
        K = sp.csr_matrix(K)
        n = M.shape[0]
        is_c = np.asarray(is_c, dtype=bool)
        is_d = ~is_c if is_d is None else np.asarray(is_d, dtype=bool)
        self.Id = np.flatnonzero(is_d)
        self.Ic = np.flatnonzero(is_c)
        self.n = n
        Mdd = M[self.Id][:, self.Id]
        if not _is_diagonal(Mdd) or M[self.Id][:, self.Ic].nnz != 0:
            raise ValueError("M^dd must be diagonal and M^dc zero (Eq. MStructure)")
        self.mdd = np.asarray(Mdd.diagonal())
        self.Kd = K[self.Id]                 # K^d = [K^dd K^dc]  (Eq. Kd)
        self.Kc = K[self.Ic]                 # K^c = [K^cd K^cc]  (Eq. Kc)
        self.fxd = np.asarray(fx)[self.Id]
        self.fxc = np.asarray(fx)[self.Ic]
        self.ft, self.dt = ft, dt
        if len(self.Ic):
            Mcc = M[self.Ic][:, self.Ic]
            Kcc = K[self.Ic][:, self.Ic]
            self.Mcc_lu = spla.splu(_csc(Mcc), permc_spec=permc_spec)
            # Calculation and factorization of the system matrix S = M^cc + beta dt^2 K^cc
            self.S_lu = spla.splu(_csc(Mcc + BETA * dt * dt * Kcc), permc_spec=permc_spec)

    def initial_state(self, u0=None, v0=None):
        """Initial acceleration for the cut DOFs and the CDM history value u^d_{-1}."""
        n, dt = self.n, self.dt
        u = np.zeros(n) if u0 is None else np.array(u0, dtype=np.float64)
        v = np.zeros(n) if v0 is None else np.asarray(v0, dtype=np.float64)
        a_c = np.zeros(n)
        if len(self.Ic):
            a_c[self.Ic] = self.Mcc_lu.solve(self.ft(0.0) * self.fxc - self.Kc @ u)
        v_c = np.zeros(n)
        v_c[self.Ic] = v[self.Ic]
        u_prev_d = np.zeros(n)
        if len(self.Id):
            a0d = (self.ft(0.0) * self.fxd - self.Kd @ u) / self.mdd
            u_prev_d[self.Id] = u[self.Id] - dt * v[self.Id] + 0.5 * dt * dt * a0d
        return ImexState(0, u, u_prev_d, v_c, a_c)

    def step(self, s):
        """One IMEX step n -> n+1 in the flowchart's order."""
        dt, Id, Ic = self.dt, self.Id, self.Ic
        t_n = s.n * dt
        t_n1 = (s.n + 1) * dt
        u = s.u
        # Diagonal CDM step
        ud_next = None
        if len(Id):
            a_d = (self.ft(t_n) * self.fxd - self.Kd @ u) / self.mdd
            ud_next = 2.0 * u[Id] - s.u_prev_d[Id] + dt * dt * a_d
        u_new = u.copy()
        u_prev_d = np.zeros(self.n)
        if len(Id):
            u_prev_d[Id] = u[Id]
            u_new[Id] = ud_next
        v_c = s.v_c.copy()
        a_c = s.a_c.copy()
        if len(Ic):
            # Prediction (u^d_pred = u^d_{n+1})
            uc_pred = u[Ic] + dt * s.v_c[Ic] + (0.5 - BETA) * dt * dt * s.a_c[Ic]
            vc_pred = s.v_c[Ic] + (1.0 - GAMMA) * dt * s.a_c[Ic]
            u_pred = u_new.copy()
            u_pred[Ic] = uc_pred
            # Acceleration calculation
            ac = self.S_lu.solve(self.ft(t_n1) * self.fxc - self.Kc @ u_pred)
            # Correction
            u_new[Ic] = uc_pred + BETA * dt * dt * ac
            v_c[Ic] = vc_pred + GAMMA * dt * ac
            a_c[Ic] = ac
        return ImexState(s.n + 1, u_new, u_prev_d, v_c, a_c)

    def run(self, nsteps, state=None, u0=None, v0=None, callback=None):
        s = self.initial_state(u0, v0) if state is None else state
        for _ in range(nsteps):
            s = self.step(s)
            if callback is not None:
                callback(s)
        return s
