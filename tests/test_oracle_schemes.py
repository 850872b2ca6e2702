"""Pins of the comparison-scheme oracle (oracle/schemes.py)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import pipeline, schemes
from oracle.discretize import CUT
from paper_2310_14712_gb300 import workloads


def _box(n=6, p=2, holes=((0.5, 0.5, 0.2, 0.2),), dt=0.0, alpha=1e-3, depth=2):
    w = workloads.Workload("box", 2, (0.0, 0.0), (1.0, 1.0), (n, n), p, alpha, depth,
                           np.asarray(holes, dtype=float).reshape(-1, 4), np.array([[0.27, 0.31]]),
                           3.0, 0.08, 0)
    w.dt = dt
    return w


def _setup(w):
    return pipeline.setup(**w.kwargs())


def test_hrz_of_a_diagonal_matrix_is_itself():
    d = np.array([0.3, 1.7, 0.02, 4.0])
    assert np.allclose(schemes.hrz_lump(np.diag(d)), np.diag(d), rtol=1e-15, atol=0)


def test_hrz_textbook_bar_elements():
    h = 0.37
    # Linear bar: consistent h/6 [[2,1],[1,2]] lumps to h/2 per node.
    lin = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    assert np.allclose(np.diag(schemes.hrz_lump(lin)), [h / 2, h / 2], rtol=1e-15, atol=0)
    # Quadratic bar: h/30 [[4,2,-1],[2,16,2],[-1,2,4]] lumps to h [1/6, 2/3, 1/6].
    quad = h / 30.0 * np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]])
    out = schemes.hrz_lump(quad)
    assert np.allclose(np.diag(out), h * np.array([1 / 6, 2 / 3, 1 / 6]), rtol=1e-14, atol=0)
    assert np.count_nonzero(out - np.diag(np.diag(out))) == 0


def test_hrz_preserves_element_mass_and_positivity():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((9, 9))
    Me = B @ B.T + 0.1 * np.eye(9)
    L = schemes.hrz_lump(Me)
    assert L.sum() == pytest.approx(Me.sum(), rel=1e-13)
    assert (np.diag(L) > 0).all()


def test_assembled_hrz_mass():
    s = _setup(_box())
    d = s.disc
    Mh = schemes.hrz_mass(s)
    M = sp.csr_matrix(d.M)
    assert sp.triu(Mh, 1).nnz == 0 and sp.tril(Mh, -1).nnz == 0
    one = np.ones(d.grid.nnodes)
    assert one @ (Mh @ one) == pytest.approx(one @ (M @ one), rel=1e-13)
    # Rows of explicit DOFs (only uncut cells around them) keep the GLL diagonal.
    Id = np.flatnonzero(d.is_d)
    assert np.allclose(Mh.diagonal()[Id], M.diagonal()[Id], rtol=1e-14, atol=0)
    assert (Mh.diagonal()[d.active] > 0).all()
    assert (d.cell_type == CUT).any()


@pytest.mark.parametrize("mass", ["consistent", "hrz"])
def test_element_eigenvalue_bound(mass):
    # Central differences are stable for dt < 2 / sqrt(lambda_max(K, M)); the
    # global lambda_max is bounded by the largest cell-wise one.
    s = _setup(_box())
    d = s.disc
    act = np.flatnonzero(d.active)
    K = sp.csr_matrix(d.K)[act][:, act].toarray()
    M = (sp.csr_matrix(d.M) if mass == "consistent" else schemes.hrz_mass(s))[act][:, act].toarray()
    lam = sla.eigh(K, M, eigvals_only=True)[-1]
    dt_u, dt_c = schemes.cellwise_critical_dt(s, mass)
    lam_cells = (2.0 / min(dt_u, dt_c)) ** 2
    assert lam <= lam_cells * (1 + 1e-10)
    assert lam >= 0.2 * lam_cells
    # The uncut value is the closed form of the time step rule.
    assert dt_u == pytest.approx(s.dt / 0.9, rel=1e-12)
    # Badly cut cells restrict the explicit step (Table criticaltimestepsizes).
    assert dt_c < dt_u


def test_without_cut_cells_all_central_difference_forms_are_imex():
    w = _box(holes=np.zeros((0, 4)))
    s = _setup(w)
    n = 60
    ref = schemes.run(s, "imex", n)
    for sch in ("cdm", "cdm_hrz"):
        st = schemes.run(s, sch, n)
        assert pipeline.relative_l2(st.u, ref.u, s.disc.active) <= 1e-13
        assert pipeline.relative_l2(st.u_prev, ref.u_prev, s.disc.active) <= 1e-13


def test_trapezoidal_is_imex_with_every_dof_implicit():
    s = _setup(_box())
    n = 40
    st = schemes.run(s, "trapezoidal", n)
    ref = schemes.imex_all_implicit(s).run(n)
    act = s.disc.active
    assert pipeline.relative_l2(st.u, ref.u, act) <= 1e-11
    assert pipeline.relative_l2(st.v, ref.v_c, act) <= 1e-10


@pytest.mark.parametrize("mass", ["consistent", "hrz"])
def test_central_differences_stable_below_critical_step_and_not_above(mass):
    w = _box(n=4, p=2)
    s0 = _setup(w)
    d = s0.disc
    act = np.flatnonzero(d.active)
    K = sp.csr_matrix(d.K)[act][:, act].toarray()
    M = (sp.csr_matrix(d.M) if mass == "consistent" else schemes.hrz_mass(s0))[act][:, act].toarray()
    lam, vec = sla.eigh(K, M)
    dt_crit = 2.0 / np.sqrt(lam[-1])
    sch = "cdm" if mass == "consistent" else "cdm_hrz"
    u0 = np.zeros(d.grid.nnodes)
    u0[act] = vec[:, -1] + 1e-3 * vec[:, len(act) // 2]
    growth = {}
    for f in (0.98, 1.02):
        w.dt = f * dt_crit
        w.src_amp = 0.0
        s = _setup(w)
        st = schemes.run(s, sch, 400, u0=u0)
        growth[f] = np.abs(st.u).max() / np.abs(u0).max()
    assert growth[0.98] < 2.0
    assert growth[1.02] > 1e3


def test_hrz_keeps_the_diagonal_shape_unlike_row_sums():
    rng = np.random.default_rng(11)
    B = rng.standard_normal((7, 7))
    Me = B @ B.T + 0.05 * np.eye(7)
    r = np.diag(schemes.hrz_lump(Me)) / np.diag(Me)
    assert np.ptp(r) <= 1e-14 * r.mean()
    # Row sums of the same matrix differ (and may be negative): not what HRZ gives.
    assert not np.allclose(Me.sum(axis=1), np.diag(schemes.hrz_lump(Me)))
