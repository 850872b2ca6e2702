"""Oracle on the plate16 workload: partition sanity and the roundoff floor that
GPU parity is judged against.

Two correct FP64 runs that differ only in the sparse ordering of the implicit
solve (SuperLU COLAMD vs natural) disagree by about 1e-11 after 500 steps, all
of it on the fictitious nodes inside the hole: there alpha = 1e-5 scales mass
and stiffness alike, S = M^cc + dt^2/4 K^cc has a condition number near 3e6,
and the weakly coupled fictitious medium keeps whatever roundoff it receives.
On physical DOFs the two agree to about 1e-14.

Summing every element quadrature in reverse point order (discretize's
quad_reverse) gives the same K and M up to about 1e-15 of max |K|; because
the fictitious entries of cut-cell matrices are alpha = 1e-5 times the
physical ones, that roundoff is a larger relative change there, and the run
drifts further from the reference than a reordering does.  Both variants
bound the rounding floor of the GPU parity tests (tests/parity_util.py).
"""
import numpy as np
import pytest

from oracle import pipeline
from oracle.geometry import Holes
from oracle.integrators import NewmarkImex
from paper_2310_14712_gb300 import workloads


def oracle_floor(s, holes, nsteps):
    """Relative L2 difference of two oracle runs (COLAMD vs natural ordering)
    on all active DOFs and on physical active DOFs."""
    d = s.disc
    alt = NewmarkImex(d.M, d.K, d.fx, s.ft, s.dt, d.is_c, d.is_d, permc_spec="NATURAL")
    a = s.imex.run(nsteps)
    b = alt.run(nsteps)
    phys = Holes(holes, s.grid.dim).physical(s.grid.node_coords()) & d.active
    return (pipeline.relative_l2(b.u, a.u, d.active), pipeline.relative_l2(b.u, a.u, phys), a)


def test_plate16_partition_and_noise_floor():
    w = workloads.plate16(steps=500)
    s = pipeline.setup(**w.kwargs())
    d = s.disc
    assert d.is_c.sum() > 0 and d.is_d.sum() > 0
    assert (d.cell_type == 2).sum() > 0                 # empty cells inside the hole are dropped
    f_all, f_phys, st = oracle_floor(s, w.holes, 500)
    assert np.linalg.norm(st.u) > 0
    assert f_phys < 1e-13, f_phys
    assert f_all < 5e-11, f_all


def test_reversed_quadrature_is_the_same_system_up_to_roundoff():
    w = workloads.plate16(steps=500)
    s = pipeline.setup(**w.kwargs())
    r = pipeline.setup(**{**s.args, "dt": s.dt}, quad_reverse=True)
    for A, B in ((s.disc.K, r.disc.K), (s.disc.M, r.disc.M)):
        scale = abs(A).max()
        assert abs(B - A).max() <= 1e-14 * scale
        assert abs(B - B.T).max() <= 1e-14 * scale
    assert np.abs(r.disc.K @ np.ones(r.disc.K.shape[0])).max() <= 1e-13 * abs(r.disc.K).max()
    assert np.abs(r.disc.fx - s.disc.fx).max() <= 1e-14 * np.abs(s.disc.fx).max()
    assert np.array_equal(r.disc.is_c, s.disc.is_c) and np.array_equal(r.disc.active, s.disc.active)
    # A correct run of the same method: physical DOFs agree like a reordering.
    a = s.imex.run(500)
    b = r.imex.run(500)
    phys = Holes(w.holes, 2).physical(s.grid.node_coords()) & s.disc.active
    assert pipeline.relative_l2(b.u, a.u, phys) < 1e-12
    assert pipeline.relative_l2(b.u, a.u, s.disc.active) < 2e-10


def test_time_step_rule_takes_the_fastest_uncut_cell():
    # dt = 0.9 * 2 / sqrt(lambda_max(K_e, M_e)) of an uncut cell at the largest
    # wave speed among uncut cells.  lambda_max grows with c^2, so a speed of 2
    # everywhere halves dt (a power of two: exactly), one uncut cell at speed 3
    # divides it by 3, and a faster cut cell does not count.
    holes = np.array([[0.5, 0.5, 0.2, 0.2]])
    kw = dict(dim=2, lo=(0, 0), hi=(1, 1), ncells=(8, 8), p=3, alpha=1e-5, depth=3, holes=holes,
              src_pos=np.array([[0.2, 0.2]]), f0=5.0, src_sigma=0.05)
    base = pipeline.setup(**kw)
    types = base.disc.cell_type
    c = np.ones(len(types))
    assert pipeline.setup(**kw, cell_c=c).dt == base.dt
    assert pipeline.setup(**kw, cell_c=2.0 * c).dt == base.dt / 2
    c[np.flatnonzero(types == 0)[5]] = 3.0
    c[np.flatnonzero(types == 1)[0]] = 5.0
    assert pipeline.setup(**kw, cell_c=c).dt == pytest.approx(base.dt / 3, rel=1e-13)


def test_independent_columns_superpose_to_the_multi_source_run():
    # The method is linear in the load (Fig. TrapCDMIMEX with f = f_t(t) f_x),
    # and a setup with several bells sums their loads, so the columns of
    # setup_columns (one source each) must add up to the run with all sources.
    holes = np.array([[0.5, 0.5, 0.2, 0.2]])
    pos = np.array([[0.2, 0.2], [0.8, 0.3], [0.25, 0.75]])
    kw = dict(dim=2, lo=(0, 0), hi=(1, 1), ncells=(8, 8), p=3, alpha=1e-5, depth=3, holes=holes,
              f0=5.0, src_sigma=0.05)
    cols = pipeline.setup_columns(pos, **kw)
    both = pipeline.setup(src_pos=pos, **kw)
    total = sum(pipeline.run(c, 60).u for c in cols)
    ref = pipeline.run(both, 60).u
    assert np.linalg.norm(ref) > 0
    assert pipeline.relative_l2(total, ref, both.disc.active) < 1e-12
    # and each column differs from the others (its own source)
    assert pipeline.relative_l2(pipeline.run(cols[1], 60).u, pipeline.run(cols[0], 60).u) > 0.5


def test_imex_stability_limit_on_the_plate_is_the_explicit_subsystems():
    # Sec. Spring-coupled masses (Fig. springCoupledMassesElastic) shows the
    # IMEX step limited by the explicit DOFs alone; the same holds on the
    # immersed plate: with the critical step of the explicit subsystem,
    # 2 / sqrt(lambda_max(K^dd, M^dd)), the potential energy u^T K u of a
    # seeded random start (no load) stays bounded over 600 steps at 0.99 of
    # it and grows without bound at 1.01.  The cell-wise step of the time
    # step rule is a lower bound of that limit (element eigenvalue bound).
    import scipy.linalg as sl
    import scipy.sparse as sp
    w = workloads.plate16()
    s = pipeline.setup(**{**w.kwargs(), "src_amp": 0.0})
    d = s.disc
    Id = np.flatnonzero(d.is_d)
    K = sp.csr_matrix(d.K)
    mdd = sp.csr_matrix(d.M)[Id][:, Id].diagonal()
    Kdd = K[Id][:, Id].toarray()
    dt_x = 2.0 / np.sqrt(sl.eigh(Kdd / np.sqrt(np.outer(mdd, mdd)), eigvals_only=True)[-1])
    dt_cell = s.dt / 0.9
    assert 0.99 * dt_x < dt_cell <= dt_x
    u0 = np.where(d.active, np.random.default_rng(3).standard_normal(len(d.active)), 0.0)
    growth = {}
    for fac in (0.99, 1.01):
        e = []
        NewmarkImex(d.M, d.K, d.fx, lambda t: 0.0, fac * dt_x, d.is_c, d.is_d).run(
            600, u0=u0, callback=lambda st: e.append(float(st.u @ (K @ st.u))))
        growth[fac] = max(e) / max(e[:50])
    assert growth[0.99] < 1.5
    assert growth[1.01] > 1e20
