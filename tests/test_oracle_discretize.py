"""Pins of the oracle's discretisation: element matrices, spacetree quadrature,
assembly invariants and the time-step rule, against values the paper prints and
against closed forms."""
import os
import numpy as np
import scipy.linalg as sl
import pytest

from oracle import discretize as D, geometry as G, pipeline, sources

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_fill():
    rows = []
    for line in open(os.path.join(GOLD, "fill_ratio_eigenfrequencies.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p, eta, om = line.split()
        rows.append((int(p), float(eta), float(om)))
    return rows


def _golden_dt():
    out = {}
    for line in open(os.path.join(GOLD, "critical_time_steps.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = float(val)
    return out


def single_cell_omega(p, eta, depth, alpha=1e-6):
    """Highest eigenfrequency of the unit cell of Fig. fillRatio cut at height eta."""
    h = np.array([1.0, 1.0])
    lo = np.zeros(2)
    if eta >= 1.0:
        Ke, Me, _ = D.uncut_element(p, h, 1.0, 1.0, lo, None)
    else:
        g = G.HalfSpace(1, eta, 2)
        xr, wr, ph = D.spacetree_points(g, lo, lo + h, depth, p, 2)
        Ke, Me, _ = D.element_from_points(p, h, xr, wr, np.where(ph, 1.0, alpha), 1.0, 1.0, None)
    return np.sqrt(sl.eigh(Ke, Me, eigvals_only=True).max())


@pytest.mark.parametrize("p,eta,omega", [r for r in _golden_fill() if r[1] in (0.0, 0.5, 1.0)])
def test_single_cell_exact_split(p, eta, omega):
    # A cut at 0 or 1/2 is resolved exactly by the first bisection, so the
    # quadtree integrates exactly and the printed value is reproduced to its digits.
    assert single_cell_omega(p, eta, 13) == pytest.approx(omega, rel=1e-9)


@pytest.mark.parametrize("p,eta,omega", [r for r in _golden_fill()
                                         if r[1] in (0.005, 0.1, 0.3, 0.74)])
def test_single_cell_quadtree_depth13(p, eta, omega):
    # Cuts that are not dyadic need the depth-13 quadtree of Fig. fillRatioHZ.
    assert single_cell_omega(p, eta, 13) == pytest.approx(omega, rel=1e-7)


def test_uncut_critical_time_step_table():
    gold = _golden_dt()
    assert D.uncut_critical_dt(5, [0.25, 0.25]) == pytest.approx(gold["uncut_p5_h0.25"], rel=1e-13)
    # Scaling: dt_crit is proportional to h / c.
    assert D.uncut_critical_dt(5, [0.125, 0.125], c=2.0) == pytest.approx(gold["uncut_p5_h0.25"] / 4, rel=1e-12)


def _small_problem(alpha=1e-5, holes=((0.5, 0.5, 0.2, 0.2),), n=8, p=3, depth=3):
    holes = np.asarray(holes, dtype=float).reshape(-1, 4)
    return pipeline.setup(2, (0, 0), (1, 1), (n, n), p, alpha, depth, holes,
                          np.array([[0.2, 0.2]]), 5.0, 0.05)


def test_assembly_invariants():
    s = _small_problem()
    d = s.disc
    K, M = d.K, d.M
    assert abs(K - K.T).max() <= 1e-13 * abs(K).max()
    ones = np.where(d.active, 1.0, 0.0)
    assert np.abs(K @ ones).max() <= 1e-12 * abs(K).max()       # constants in the null space (Neumann)
    # 1^T M 1 equals the alpha-weighted quadrature volume, cell by cell.
    area = np.prod(d.grid.h)
    vol = 0.0
    for cid, t in enumerate(d.cell_type):
        if t == G.UNCUT:
            vol += area
        elif t == G.CUT:
            vol += area * (d.fill[cid] + d.alpha * (1.0 - d.fill[cid]))
    assert ones @ (M @ ones) == pytest.approx(vol, rel=1e-13)
    # Partition (Eq. MStructure): M^dd diagonal and positive, M^dc = 0.
    Id, Ic = np.flatnonzero(d.is_d), np.flatnonzero(d.is_c)
    Mdd = M[Id][:, Id].tocoo()
    assert np.all(Mdd.row == Mdd.col) and np.all(Mdd.data > 0)
    assert M[Id][:, Ic].nnz == 0
    assert not (d.is_d & d.is_c).any()


def test_physical_area_converges_to_analytic():
    # Physical area = box - circle, recovered by the quadtree within its resolution.
    errs = []
    for depth in (2, 4, 6):
        s = _small_problem(alpha=1e-12, depth=depth, p=2)
        d = s.disc
        area = np.prod(d.grid.h)
        phys = sum(area * (d.fill[c] if t == G.CUT else 1.0)
                   for c, t in enumerate(d.cell_type) if t != G.EMPTY)
        errs.append(abs(phys - (1.0 - np.pi * 0.2 ** 2)))
    assert errs[2] < errs[0] / 8 and errs[2] < 2e-4


def _standing_mode_error(n, p, hole_r, dt_scale=1.0, t_end=1.0):
    """alpha = 1 everywhere: the box problem has the exact solution
    cos(pi x) cos(pi y) cos(sqrt(2) pi t) for Neumann walls and f = 0."""
    holes = np.array([[0.5, 0.5, hole_r, hole_r]]) if hole_r > 0 else np.zeros((0, 4))
    s = pipeline.setup(2, (0, 0), (1, 1), (n, n), p, 1.0, 3, holes,
                       np.array([[0.2, 0.2]]), 5.0, 0.05, src_amp=0.0)
    dt0 = s.dt * dt_scale
    nsteps = int(round(t_end / dt0))
    dt = t_end / nsteps
    from oracle.integrators import NewmarkImex
    imex = NewmarkImex(s.disc.M, s.disc.K, s.disc.fx, lambda t: 0.0, dt, s.disc.is_c, s.disc.is_d)
    X = s.grid.node_coords()
    u0 = np.cos(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    st = imex.run(nsteps, u0=u0)
    exact = u0 * np.cos(np.sqrt(2.0) * np.pi * t_end)
    s.u_final, s.u0, s.nsteps, s.dt_used = st.u, u0, nsteps, dt
    return pipeline.relative_l2(st.u, exact, s.disc.active), s


def test_standing_mode_all_uncut():
    err, s = _standing_mode_error(8, 4, 0.0)
    assert not s.disc.is_c.any()
    # Against the PDE: only the CDM phase error omega^3 dt^2 t / 24 (about 5e-4
    # rad here, divided by |cos(omega T)| = 0.27) remains.
    assert err < 2.5e-3
    # Against the exact discrete CDM solution cos(n theta) u0, cos(theta) =
    # 1 - lambda dt^2 / 2 with lambda = 2 pi^2: only the spatial error remains.
    theta = np.arccos(1.0 - np.pi ** 2 * s.dt_used ** 2)
    err_d = pipeline.relative_l2(s.u_final, s.u0 * np.cos(s.nsteps * theta), s.disc.active)
    assert err_d < 1e-6


def test_standing_mode_with_cut_cells():
    # A hole with alpha_f = 1 only changes the quadrature (cut cells get the
    # consistent spacetree mass and go to the implicit partition): the exact
    # solution is unchanged.
    err, s = _standing_mode_error(8, 4, 0.13)
    assert s.disc.is_c.sum() > 50 and s.disc.is_d.sum() > 50
    assert err < 2.5e-3


def test_standing_mode_second_order_in_time():
    e1, _ = _standing_mode_error(6, 5, 0.13, dt_scale=1.0)
    e2, _ = _standing_mode_error(6, 5, 0.13, dt_scale=0.5)
    assert 3.3 < e1 / e2 < 4.5


def _load_sum(grid, geom, alpha, depth, f):
    d = D.discretize(grid, geom, alpha, depth, fx=f)
    return d, float(d.fx.sum())


def test_load_vector_integrates_constant_and_linear_loads():
    # Eq. f with the basis summing to one: sum_i f_i = int alpha f.  Without
    # holes that is a closed form (GL integrates f exactly); the box does not
    # start at the origin, so a wrong map from reference to physical points
    # shows.  With holes the same quadrature gives 1^T M u / rho for u the
    # nodal values of f (f in the span of the basis; uncut cells: GL load and
    # GLL mass are both exact for degree 1; cut cells share M's points).
    lin = lambda x: x[:, 0] + 2.0 * x[:, 1]
    one = lambda x: np.ones(len(x))
    grid = D.Grid((0.5, 0.0), (1.5, 1.0), (4, 3), 3)
    none = G.Holes(np.zeros((0, 4)), 2)
    assert _load_sum(grid, none, 1e-5, 3, one)[1] == pytest.approx(1.0, rel=1e-13)
    # int x0 + 2 x1 over [0.5, 1.5] x [0, 1] = (1.5^2 - 0.5^2) / 2 + 2 * 1/2
    assert _load_sum(grid, none, 1e-5, 3, lin)[1] == pytest.approx(2.0, rel=1e-13)
    grid = D.Grid((0.5, 0.0), (1.5, 1.0), (8, 8), 3)
    holes = G.Holes(np.array([[1.0, 0.5, 0.23, 0.17], [0.62, 0.2, 0.1, 0.1]]), 2)
    X = grid.node_coords()
    for f in (one, lin):
        d, total = _load_sum(grid, holes, 1e-5, 3, f)
        assert (d.cell_type == G.CUT).sum() > 10
        u = np.where(d.active, f(X), 0.0)
        assert total == pytest.approx(float(np.ones(len(X)) @ (d.M @ u)), rel=1e-12)


def test_empty_cell_threshold_is_fill_ratio_1e_10():
    # Sec. 2D example: a cell whose fill ratio is below 1e-10 is discarded.
    # One 1D cell of unit length cut by the half-space x < eta: a binary tree
    # of depth 34 puts the boundary in a leaf of length 2^-34 (5.8e-11), so
    # the quadrature fill is eta to within that.
    grid = D.Grid((0.0,), (1.0,), (1,), 2)
    kept = D.discretize(grid, G.HalfSpace(0, 5e-10, 1), 1e-5, 34)
    assert kept.cell_type[0] == G.CUT and abs(kept.fill[0] - 5e-10) < 6e-11
    assert kept.active.all()
    dropped = D.discretize(grid, G.HalfSpace(0, 2e-11, 1), 1e-5, 34)
    assert dropped.cell_type[0] == G.EMPTY and dropped.fill[0] < 1e-10
    assert not dropped.active.any()


def test_stiffness_scales_with_the_square_of_the_wave_speed():
    # Eq. K carries rho c^2 and Eq. Mglobal none: a wave speed of 2 in every
    # cell, given per cell or as c0, multiplies K by 4 (exactly: a power of
    # two) and leaves M alone, on uncut and cut cells alike.
    grid = D.Grid((0.0, 0.0), (1.0, 1.0), (6, 6), 3)
    holes = G.Holes(np.array([[0.5, 0.5, 0.2, 0.2]]), 2)
    one = D.discretize(grid, holes, 1e-5, 3)
    per_cell = D.discretize(grid, holes, 1e-5, 3, cell_c=np.full(36, 2.0))
    as_c0 = D.discretize(grid, holes, 1e-5, 3, c0=2.0)
    assert (one.cell_type == G.CUT).sum() > 5 and (one.cell_type == G.UNCUT).sum() > 5
    for d in (per_cell, as_c0):
        assert abs(d.K - 4.0 * one.K).max() == 0.0
        assert abs(d.M - one.M).max() == 0.0
