"""Pins of the oracle's time integrators (Sec. Time integration) to closed forms
and to the ten spring-coupled masses of Sec. "Spring-coupled masses"."""
import os
import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp
import pytest

from oracle.integrators import cdm, trapezoidal_newmark, NewmarkImex

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    for line in open(os.path.join(GOLD, "critical_time_steps.txt")):
        if line.startswith(name + " "):
            return float(line.split()[1])
    raise KeyError(name)


def _random_spd_system(n, rng, diag_mass=True):
    A = rng.standard_normal((n, n))
    K = A @ A.T + n * np.eye(n)
    if diag_mass:
        M = np.diag(rng.uniform(0.5, 2.0, n))
    else:
        B = rng.standard_normal((n, n))
        M = B @ B.T + n * np.eye(n)
    return M, K


def _mode(M, K, which):
    lam, V = sl.eigh(K, M)
    return lam[which], V[:, which]


def test_cdm_single_mode_closed_form():
    rng = np.random.default_rng(1)
    M, K = _random_spd_system(6, rng, diag_mass=False)
    lam, phi = _mode(M, K, -1)
    dt = 0.9 * 2.0 / np.sqrt(lam)
    n = 37
    u, _ = cdm(sp.csr_matrix(M), sp.csr_matrix(K), np.zeros(6), lambda t: 0.0, dt, n, phi, np.zeros(6))
    theta = np.arccos(1.0 - lam * dt * dt / 2.0)
    assert np.allclose(u, np.cos(n * theta) * phi, atol=1e-11 * np.abs(phi).max())


def test_trapezoidal_single_mode_closed_form():
    rng = np.random.default_rng(2)
    M, K = _random_spd_system(6, rng, diag_mass=False)
    lam, phi = _mode(M, K, -1)
    dt = 7.0 / np.sqrt(lam)                        # far beyond any explicit limit
    n = 23
    u, v, a = trapezoidal_newmark(sp.csr_matrix(M), sp.csr_matrix(K), np.zeros(6), lambda t: 0.0,
                                  dt, n, phi, np.zeros(6))
    q = lam * dt * dt / 4.0
    theta = np.arccos((1.0 - q) / (1.0 + q))
    assert np.allclose(u, np.cos(n * theta) * phi, atol=1e-11 * np.abs(phi).max())


def test_imex_with_no_implicit_dofs_is_cdm():
    rng = np.random.default_rng(3)
    M, K = _random_spd_system(7, rng, diag_mass=True)
    lam, phi = _mode(M, K, -2)
    dt = 0.8 * 2.0 / np.sqrt(_mode(M, K, -1)[0])
    n = 41
    imex = NewmarkImex(sp.csr_matrix(M), sp.csr_matrix(K), np.zeros(7), lambda t: 0.0, dt,
                       np.zeros(7, dtype=bool))
    st = imex.run(n, u0=phi)
    theta = np.arccos(1.0 - lam * dt * dt / 2.0)
    assert np.allclose(st.u, np.cos(n * theta) * phi, atol=1e-11 * np.abs(phi).max())


def test_imex_with_all_dofs_implicit_is_trapezoidal():
    rng = np.random.default_rng(4)
    M, K = _random_spd_system(7, rng, diag_mass=False)
    lam, phi = _mode(M, K, -1)
    dt = 5.0 / np.sqrt(lam)
    n = 29
    imex = NewmarkImex(sp.csr_matrix(M), sp.csr_matrix(K), np.zeros(7), lambda t: 0.0, dt,
                       np.ones(7, dtype=bool))
    st = imex.run(n, u0=phi)
    q = lam * dt * dt / 4.0
    theta = np.arccos((1.0 - q) / (1.0 + q))
    assert np.allclose(st.u, np.cos(n * theta) * phi, atol=1e-11 * np.abs(phi).max())


def test_imex_on_decoupled_blocks_is_cdm_plus_trapezoidal():
    # K block diagonal between I_d and I_c: each partition follows its own closed form.
    rng = np.random.default_rng(5)
    Md, Kd = _random_spd_system(4, rng, diag_mass=True)
    Mc, Kc = _random_spd_system(3, rng, diag_mass=False)
    M = sl.block_diag(Md, Mc)
    K = sl.block_diag(Kd, Kc)
    is_c = np.array([0, 0, 0, 0, 1, 1, 1], dtype=bool)
    lam_d, phi_d = _mode(Md, Kd, -1)
    lam_c, phi_c = _mode(Mc, Kc, -1)
    dt = 0.9 * 2.0 / np.sqrt(lam_d)
    u0 = np.concatenate([phi_d, phi_c])
    n = 31
    st = NewmarkImex(sp.csr_matrix(M), sp.csr_matrix(K), np.zeros(7), lambda t: 0.0, dt, is_c).run(n, u0=u0)
    th_d = np.arccos(1.0 - lam_d * dt * dt / 2.0)
    q = lam_c * dt * dt / 4.0
    th_c = np.arccos((1.0 - q) / (1.0 + q))
    assert np.allclose(st.u[:4], np.cos(n * th_d) * phi_d, atol=1e-11)
    assert np.allclose(st.u[4:], np.cos(n * th_c) * phi_c, atol=1e-11)


# ---- ten spring-coupled masses (Sec. Spring-coupled masses) ----------------------

def spring_chain():
    """Masses 1..8 = 1 kg, 9..10 = 1e-3 kg, springs k = 1 N/m; mass 1 tied to a wall,
    mass 10 free (the boundary conditions that reproduce the printed critical steps)."""
    m = np.array([1.0] * 8 + [1e-3] * 2)
    n = 10
    K = np.zeros((n, n))
    for i in range(n - 1):
        K[i, i] += 1.0
        K[i + 1, i + 1] += 1.0
        K[i, i + 1] -= 1.0
        K[i + 1, i] -= 1.0
    K[0, 0] += 1.0
    f = np.zeros(n)
    f[7] = 1.0                                          # third-last mass
    return np.diag(m), K, f


def test_spring_chain_critical_steps():
    M, K, _ = spring_chain()
    lam = sl.eigh(K, M, eigvals_only=True).max()
    assert 2.0 / np.sqrt(lam) == pytest.approx(_gold("spring_global"), rel=2e-7)
    lam_d = sl.eigh(K[:8, :8], M[:8, :8], eigvals_only=True).max()
    assert 2.0 / np.sqrt(lam_d) == pytest.approx(_gold("spring_explicit"), rel=2e-8)


def _spring_imex_error(nsteps, T=50.0, fs=0.1):
    M, K, f = spring_chain()
    w = 2.0 * np.pi * fs
    amp = np.linalg.solve(K - w * w * M, f)            # Helmholtz amplitude vector
    is_c = np.zeros(10, dtype=bool)
    is_c[8:] = True
    dt = T / nsteps
    st = NewmarkImex(sp.csr_matrix(M), sp.csr_matrix(K), f, lambda t: np.sin(w * t), dt,
                     is_c).run(nsteps, u0=np.zeros(10), v0=w * amp)
    return np.linalg.norm(st.u - amp * np.sin(w * T))


def test_spring_chain_imex_second_order():
    errs = [_spring_imex_error(n) for n in (200, 400, 800)]
    assert 3.8 < errs[0] / errs[1] < 4.2
    assert 3.8 < errs[1] / errs[2] < 4.2


def _spring_energy(dt_factor, nsteps=400):
    M, K, f = spring_chain()
    w = 2.0 * np.pi * 0.1
    amp = np.linalg.solve(K - w * w * M, f)
    is_c = np.zeros(10, dtype=bool)
    is_c[8:] = True
    dt = dt_factor * _gold("spring_explicit")
    energy = []
    NewmarkImex(sp.csr_matrix(M), sp.csr_matrix(K), f, lambda t: np.sin(w * t), dt, is_c).run(
        nsteps, u0=np.zeros(10), v0=w * amp,
        callback=lambda s: energy.append(0.5 * s.u @ K @ s.u))
    return np.asarray(energy)


def test_spring_chain_stability_limit_is_explicit_subsystem():
    # Fig. springCoupledMassesElastic: bounded at 0.99 dt_crit^explicit, growing at 1.01.
    e_ok = _spring_energy(0.99)
    e_bad = _spring_energy(1.01)
    assert e_ok.max() < 100.0 * e_ok[:50].max()
    assert e_bad[-1] > 1e6 * e_bad[:50].max()
