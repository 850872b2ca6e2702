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
