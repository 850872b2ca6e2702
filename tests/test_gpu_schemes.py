"""GPU parity of the paper's comparison schemes (central differences with the
consistent and the HRZ-lumped cut-cell masses, trapezoidal Newmark) against
the oracle (oracle/schemes.py), through the C-ABI.

Gates as for the method (tests/parity_util.py): physical DOFs relative L2
<= 1e-11; the per-node max over physical DOFs and all active DOFs within
FLOOR_FACTOR x the rounding floor (oracle runs with other sparse orderings,
and with reversed quadrature sums), at least 1e-11."""
import dataclasses

import numpy as np
import pytest

from oracle import pipeline, schemes
from paper_2310_14712_gb300 import workloads

from parity_util import FLOOR_FACTOR, ORDERINGS, phys_mask, reversed_quadrature_setup, _maxabs

pytestmark = pytest.mark.gpu


def _imex():
    from paper_2310_14712_gb300 import imex
    return imex


def _gpu_run(w, scheme, nsteps, u0=None):
    imex = _imex()
    with imex.Imex.from_workload(w, scheme=scheme) as g:
        if u0 is not None:
            g.set_initial(u0)
        g.step(nsteps)
        st = {k: g.fields(k, out=np.zeros(g.n_nodes)) for k in ("u", "u_prev_d", "v_c", "a_c")}
        info = g.info()
    return st, info


def _floor(s, scheme, nsteps, ref, u0, phys):
    # Rounding floor (tests/parity_util.py): other sparse orderings and the
    # system assembled with reversed quadrature sums; (all active, max phys).
    alts = [schemes.run(s, scheme, nsteps, u0=u0, permc_spec=spec) for spec in ORDERINGS]
    alts.append(schemes.run(reversed_quadrature_setup(s), scheme, nsteps, u0=u0))
    return (max(pipeline.relative_l2(a.u, ref.u, s.disc.active) for a in alts),
            max(_maxabs(a.u, ref.u, phys) for a in alts))


def _check(w, scheme, nsteps, u0=None):
    st, info = _gpu_run(w, scheme, nsteps, u0)
    w2 = dataclasses.replace(w, dt=info["dt"])
    s = pipeline.setup(**w2.kwargs())
    ref = schemes.run(s, scheme, nsteps, u0=u0)
    act = s.disc.active
    phys = phys_mask(s, w.holes)
    e_phys = pipeline.relative_l2(st["u"], ref.u, phys)
    e_all = pipeline.relative_l2(st["u"], ref.u, act)
    fl_all, fl_max = _floor(s, scheme, nsteps, ref, u0, phys)
    tol_all = max(1e-11, FLOOR_FACTOR * fl_all)
    assert e_phys <= 1e-11, (e_phys, e_all)
    assert _maxabs(st["u"], ref.u, phys) <= max(1e-11, FLOOR_FACTOR * fl_max)
    assert e_all <= tol_all, (e_all, tol_all)
    if ref.u_prev is not None:
        assert pipeline.relative_l2(st["u_prev_d"], ref.u_prev, phys) <= 1e-11
    if ref.v is not None:
        assert pipeline.relative_l2(st["v_c"], ref.v, phys) <= 1e-10
        assert pipeline.relative_l2(st["a_c"], ref.a, phys) <= 1e-10
    return s, info


def _standing(w):
    s = pipeline.setup(**w.kwargs())
    X = s.grid.node_coords()
    return np.cos(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])


@pytest.mark.parametrize("scheme", ["cdm", "cdm_hrz"])
def test_central_difference_time_step_is_the_cellwise_minimum(scheme):
    w = workloads.plate16()
    _, info = _gpu_run(w, scheme, 0)
    s = pipeline.setup(**w.kwargs())
    dt_u, dt_c = schemes.cellwise_critical_dt(s, "consistent" if scheme == "cdm" else "hrz")
    assert info["scheme"] == _imex().SCHEMES[scheme]
    assert info["dt_crit_uncut"] == pytest.approx(dt_u, rel=1e-12)
    assert info["dt_crit_cut_min"] == pytest.approx(dt_c, rel=1e-10)
    assert info["dt"] == pytest.approx(0.9 * min(dt_u, dt_c), rel=1e-10)


@pytest.mark.parametrize("scheme", ["cdm", "cdm_hrz", "trapezoidal"])
def test_schemes_plate16_match_oracle(scheme):
    w = workloads.plate16()
    s, info = _check(w, scheme, 300, u0=_standing(w))
    if scheme == "trapezoidal":
        assert info["n_d"] == 0 and info["n_c"] == int(s.disc.active.sum())
    else:
        assert info["n_d"] > 0 and info["n_c"] > 0


@pytest.mark.parametrize("scheme", ["cdm", "cdm_hrz", "trapezoidal"])
@pytest.mark.parametrize("p", [2, 5])
def test_schemes_ragged_grid(scheme, p):
    w = workloads.Workload("box", 2, (0.0, 0.0), (1.3, 0.7), (13, 7), p, 1e-5, 3,
                           np.array([[0.55, 0.45, 0.21, 0.21]]), np.array([[0.23, 0.31]]), 3.0, 0.08, 0)
    _check(w, scheme, 60)


def test_central_differences_without_cut_cells_are_imex_bitwise():
    w = workloads.Workload("box", 2, (0.0, 0.0), (1.0, 1.0), (9, 9), 4, 1e-5, 3,
                           np.zeros((0, 4)), np.array([[0.23, 0.31]]), 3.0, 0.08, 0)
    ref, _ = _gpu_run(w, "imex", 80)
    for scheme in ("cdm", "cdm_hrz"):
        st, info = _gpu_run(w, scheme, 80)
        assert info["n_c"] == 0
        assert np.array_equal(st["u"], ref["u"]) and np.array_equal(st["u_prev_d"], ref["u_prev_d"])


@pytest.mark.parametrize("scheme", ["cdm_hrz", "trapezoidal"])
def test_schemes_with_independent_columns(scheme):
    imex = _imex()
    w = workloads.multisource(nsrc=3)
    n = 80
    with imex.Imex.from_workload(w, ncols=3, scheme=scheme) as g:
        g.step(n)
        u = g.fields("u", out=np.zeros(g.field_len)).reshape(3, -1)
        dt = g.info()["dt"]
    kw = w.kwargs()
    pos = kw.pop("src_pos")
    kw["dt"] = dt
    for k, s in enumerate(pipeline.setup_columns(pos, **kw)):
        ref = schemes.run(s, scheme, n)
        assert pipeline.relative_l2(u[k], ref.u, phys_mask(s, w.holes)) <= 1e-11


def test_scheme_restrictions():
    imex = _imex()
    w = workloads.plate16()
    with imex.Imex.from_workload(w, scheme="cdm") as g:
        with pytest.raises(imex.ImexError):
            g.set_solver("pcg_jacobi")
        with pytest.raises(imex.ImexError):
            g.adjoint(4, np.array([5]), np.zeros((4, 1, 1)))


def test_health_check_reports_divergence_above_the_critical_step():
    # Central differences at 1.5 x the global critical step of a small plate
    # grow by about 2x per step until the state overflows; the health check
    # reports it (IMEX_ERR_DIVERGED).  Below the step it returns max |u|.
    import scipy.linalg as sla
    import scipy.sparse as sp
    imex = _imex()
    w = workloads.Workload("box", 2, (0.0, 0.0), (1.0, 1.0), (4, 4), 2, 1e-3, 2,
                           np.array([[0.5, 0.5, 0.2, 0.2]]), np.array([[0.27, 0.31]]), 3.0, 0.08, 0)
    s = pipeline.setup(**w.kwargs())
    act = np.flatnonzero(s.disc.active)
    K = sp.csr_matrix(s.disc.K)[act][:, act].toarray()
    M = sp.csr_matrix(s.disc.M)[act][:, act].toarray()
    dt_crit = 2.0 / np.sqrt(sla.eigh(K, M, eigvals_only=True)[-1])
    X = s.grid.node_coords()
    u0 = np.cos(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    stable = dataclasses.replace(w, dt=0.9 * dt_crit)
    with imex.Imex.from_workload(stable, scheme="cdm") as g:
        g.set_initial(u0)
        g.step(300)
        u = g.fields("u", out=np.zeros(g.n_nodes))
        assert g.check_finite() == pytest.approx(np.abs(u[s.disc.active]).max(), rel=0, abs=0)
    unstable = dataclasses.replace(w, dt=1.5 * dt_crit)
    with imex.Imex.from_workload(unstable, scheme="cdm") as g:
        g.set_initial(u0)
        g.step(20)
        assert np.isfinite(g.check_finite())
        g.step(3000)
        with pytest.raises(imex.ImexError, match="DIVERGED"):
            g.check_finite()


@pytest.mark.parametrize("scheme", ["cdm", "cdm_hrz", "trapezoidal"])
def test_schemes_3d(scheme):
    # 4 x 3 x 3 cells, p = 2, one ellipsoidal void, octree depth 2.
    w = workloads.Workload("box3", 3, (0.0, 0.0, 0.0), (1.0, 0.8, 0.6), (4, 3, 3), 2, 1e-5, 2,
                           np.array([[0.55, 0.4, 0.3, 0.22, 0.18, 0.15]]), np.array([[0.21, 0.27, 0.22]]),
                           3.0, 0.1, 0)
    _check(w, scheme, 40)


def test_trapezoidal_with_large_supernodes():
    # Every active DOF implicit on a 96 x 48-cell perforated plate (p = 4, the
    # 24 seeded holes): 70k implicit DOFs whose top dissection supernodes carry
    # more than 256 ancestor rows, walked as row chunks over many CTAs.
    w = workloads.plate256()
    w.ncells = (96, 48)
    s, info = _check(w, "trapezoidal", 100)
    assert info["large_supernodes"] > 0 and info["max_rows"] > 256
    assert info["n_d"] == 0
