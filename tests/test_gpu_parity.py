"""GPU parity: the CUDA path (through the C-ABI) against the FP64 CPU oracle.

Tolerances (tests/parity_util.py)
  * physical DOFs: relative L2 <= 1e-11 after the full step count, and the
    per-node max |u - u_ref| over physical DOFs <= max(1e-11, FLOOR_FACTOR x
    its rounding floor) x max |u_ref|;
  * all active DOFs: relative L2 <= max(1e-11, FLOOR_FACTOR x floor), the
    floor being the largest disagreement between the reference oracle run and
    oracle runs that evaluate the method in another correct FP64 way (other
    sparse orderings; every element quadrature summed in reverse order),
    measured here per case.  The floor comes from the fictitious nodes inside
    holes (alpha = 1e-5 makes S = M^cc + dt^2/4 K^cc ill-conditioned);
  * one step from a given state, and the initial state: <= 1e-13.
"""
import types

import numpy as np
import pytest

from oracle import pipeline
from oracle.geometry import Holes
from oracle.integrators import NewmarkImex
from paper_2310_14712_gb300 import workloads

from parity_util import Floor, check_state, parallel_reference_and_floor, phys_mask

pytestmark = pytest.mark.gpu


def _imex():
    # Import here so that a missing extension fails the GPU tests loudly.
    from paper_2310_14712_gb300 import imex
    return imex


def _kw(w):
    return w.kwargs()


def _gpu_state(g):
    return {k: g.fields(k, out=np.zeros(g.n_nodes)) for k in ("u", "u_prev_d", "v_c", "a_c")}


def _phys_mask(s, holes):
    return Holes(holes, s.grid.dim).physical(s.grid.node_coords()) & s.disc.active


def _check_run(w, nsteps, u0=None, v0=None, use_floor=True):
    imex = _imex()
    s = pipeline.setup(**_kw(w))
    ref = s.imex.run(nsteps, u0=u0, v0=v0)
    with imex.Imex.from_workload(w) as g:
        if u0 is not None:
            g.set_initial(u0, v0)
        g.step(nsteps)
        st = _gpu_state(g)
        info = g.info()
    assert info["step"] == nsteps
    e_phys, e_all = check_state(s, ref, st, w.holes, w.alpha, nsteps, use_floor, u0, v0)
    return e_phys, e_all, info


def test_initial_state_matches_oracle():
    imex = _imex()
    w = workloads.plate16()
    s = pipeline.setup(**_kw(w))
    ref = s.imex.initial_state()
    with imex.Imex.from_workload(w) as g:
        st = _gpu_state(g)
    d = s.disc
    assert np.array_equal(st["u"], np.zeros_like(st["u"]))
    assert pipeline.relative_l2(st["u_prev_d"], ref.u_prev_d, d.is_d) <= 1e-13
    # a^c_0 solves with M^cc, whose consistent alpha-scaled cut-cell blocks make
    # it far worse conditioned than S: judge it against the oracle's own floor.
    alt = NewmarkImex(d.M, d.K, d.fx, s.ft, s.dt, d.is_c, d.is_d, permc_spec="NATURAL").initial_state()
    floor = pipeline.relative_l2(alt.a_c, ref.a_c, d.is_c)
    phys = _phys_mask(s, w.holes) & d.is_c
    assert pipeline.relative_l2(st["a_c"], ref.a_c, phys) <= 1e-12
    assert pipeline.relative_l2(st["a_c"], ref.a_c, d.is_c) <= max(1e-12, 10.0 * floor)


@pytest.mark.parametrize("nsteps", [1, 3, 20])
def test_first_steps_plate16(nsteps):
    _check_run(workloads.plate16(), nsteps)


def test_plate16_full_500_steps():
    e_phys, e_all, info = _check_run(workloads.plate16(steps=500), 500)
    assert info["n_c"] > 0 and info["n_d"] > 0


def test_masks_and_load_vector():
    imex = _imex()
    w = workloads.plate16()
    s = pipeline.setup(**_kw(w))
    with imex.Imex.from_workload(w) as g:
        md = g.fields("mask_d", out=np.zeros(g.n_nodes))
        mc = g.fields("mask_c", out=np.zeros(g.n_nodes))
        fx = g.fields("fx", out=np.zeros(g.n_nodes))
    assert np.array_equal(md > 0, s.disc.is_d)
    assert np.array_equal(mc > 0, s.disc.is_c)
    assert np.abs(fx - s.disc.fx).max() <= 1e-13 * np.abs(s.disc.fx).max()


def _box(n, p, holes, alpha=1e-5, depth=3, ncy=None, lo=(0.0, 0.0), hi=(1.0, 1.0)):
    return workloads.Workload("box", 2, lo, hi, (n, ncy or n), p, alpha, depth,
                              np.asarray(holes, dtype=float).reshape(-1, 4),
                              np.array([[0.23, 0.31]]), 3.0, 0.08, 0)


@pytest.mark.parametrize("variant", ["large", "sweep", "sweep_short", "small_split2"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_orders_ragged_grid(p, variant, monkeypatch):
    # 13 x 7 cells: not a multiple of any tile or strip width; one hole
    # crossing the top edge.  Every explicit form (tiles; the strip sweep with
    # 3 CTAs, whose unit ranges start mid-strip and cross strips; small tiles
    # with the split launch beside the solve).
    monkeypatch.setenv("IMEX_EXPLICIT_TILE", variant)
    if variant.startswith("sweep"):
        monkeypatch.setenv("IMEX_SWEEP_CTAS", "3")
    w = _box(13, p, [[0.55, 0.62, 0.21, 0.21]], ncy=7, hi=(1.3, 0.7))
    e_phys, e_all, info = _check_run(w, 40)
    assert info["n_c"] > 0


def test_no_holes_all_explicit():
    w = _box(9, 4, np.zeros((0, 4)))
    e_phys, e_all, info = _check_run(w, 60)
    assert info["n_c"] == 0


def test_all_cells_cut_all_implicit():
    # 2 x 2 cells around one hole: every cell is cut, I_d is empty (pure trapezoidal).
    w = _box(2, 3, [[0.5, 0.5, 0.3, 0.3]])
    e_phys, e_all, info = _check_run(w, 50)
    assert info["n_d"] == 0


def test_many_holes_and_components():
    w = workloads.plate256()
    w.ncells = (48, 24)
    w.p = 3
    e_phys, e_all, info = _check_run(w, 100)
    assert info["n_components"] > 5


def test_multilevel_solve_schedule():
    # A 6 x 6 lattice of holes (r = 0.07) on 16 x 16 cells, p = 4: one implicit
    # component of about 4000 DOFs whose dissection tree is walked in several
    # launches per direction below the dense top (descendant updates gathered
    # across launches).
    centres = (np.arange(6) + 0.5) / 6.0
    w = _box(16, 4, [[x, y, 0.07, 0.07] for x in centres for y in centres])
    e_phys, e_all, info = _check_run(w, 100)
    assert info["solve_levels"] >= 2


def test_standing_mode_against_oracle_and_closed_form():
    # alpha = 1 everywhere: u = cos(pi x) cos(pi y) cos(sqrt(2) pi t) on the box.
    w = _box(8, 4, [[0.5, 0.5, 0.13, 0.13]], alpha=1.0)
    w.src_amp = 0.0
    s = pipeline.setup(**_kw(w))
    X = s.grid.node_coords()
    u0 = np.cos(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    e_phys, e_all, info = _check_run(w, 82, u0=u0)
    imex = _imex()
    with imex.Imex.from_workload(w) as g:
        g.set_initial(u0)
        g.step(82)
        u = g.fields("u", out=np.zeros(g.n_nodes))
        dt = g.info()["dt"]
    exact = u0 * np.cos(np.sqrt(2.0) * np.pi * 82 * dt)
    assert pipeline.relative_l2(u, exact, s.disc.active) < 2.5e-3


def test_checkpoint_resume_is_bit_exact():
    imex = _imex()
    w = workloads.plate16()
    with imex.Imex.from_workload(w) as a:
        a.step(30)
        ck = _gpu_state(a)
        a.step(25)
        ua = a.fields("u", out=np.zeros(a.n_nodes))
    with imex.Imex.from_workload(w) as b:
        for k, v in ck.items():
            b.set_fields(k, v)
        b.set_step(30)
        b.step(25)
        ub = b.fields("u", out=np.zeros(b.n_nodes))
    assert np.array_equal(ua, ub)


def test_deterministic_runs():
    imex = _imex()
    w = workloads.plate16()
    outs = []
    for _ in range(2):
        with imex.Imex.from_workload(w) as g:
            g.step(40)
            outs.append(g.fields("u", out=np.zeros(g.n_nodes)))
    assert np.array_equal(outs[0], outs[1])


def test_plate256_full_5000_steps():
    # The benchmarked workload (256 x 128 cells, p = 4, 24 holes) for its full
    # 5000 steps on every node; the reference and the four floor variants run
    # in parallel worker processes while the device steps.
    import concurrent.futures as cf
    w = workloads.plate256()
    imex = _imex()
    with imex.Imex.from_workload(w) as g:
        dt = g.info()["dt"]
        with cf.ThreadPoolExecutor(1) as pool:
            # dt = w.dt (0: the oracle's own 0.9 x uncut critical step)
            fut = pool.submit(parallel_reference_and_floor, _kw(w), w.dt, w.steps)
            g.step(w.steps)
            st = _gpu_state(g)
            ref_f, variants = fut.result()
        info = g.info()
    assert info["step"] == w.steps
    s = pipeline.setup(**_kw(w))
    assert s.dt == pytest.approx(dt, rel=1e-14)
    ref = types.SimpleNamespace(**ref_f)
    fl = Floor()
    for name, v in variants.items():
        fl.add(name, v["u"], ref.u, s, w.holes)
    e_phys, e_all = check_state(s, ref, st, w.holes, w.alpha, w.steps, floor=fl)
    assert np.abs(ref.u[phys_mask(s, w.holes)]).max() > 1e-6   # the pulse has crossed the plate


def test_step_io_source_samples_and_receivers():
    # User-supplied source samples replace f_t for the steps; receiver traces
    # equal u at the receiver nodes after every step.  The initial state (set up
    # with the built-in wavelet's f_t(0)) is the same on both sides, so sample 0
    # is that value.
    imex = _imex()
    w = workloads.plate16()
    s = pipeline.setup(**_kw(w))
    n = 60
    sig = workloads.source_signature(n + 1, s.dt)
    sig[0] = s.ft(0.0)
    rec = workloads.receiver_nodes(w, 16)
    st0 = s.imex.initial_state()
    s.imex.ft = lambda t: float(sig[int(round(t / s.dt))])
    traces_ref = np.zeros((n, len(rec)))

    def cb(st):
        traces_ref[st.n - 1] = st.u[rec]

    ref = s.imex.run(n, state=st0, callback=cb)
    with imex.Imex.from_workload(w) as g:
        traces = np.zeros((n, len(rec)))
        g.step_io(n, sig, rec, traces)
        u = g.fields("u", out=np.zeros(g.n_nodes))
    assert pipeline.relative_l2(u, ref.u, _phys_mask(s, w.holes)) <= 1e-11
    assert np.abs(traces - traces_ref).max() <= 1e-11 * np.abs(ref.u).max()
    assert np.array_equal(traces[-1], u[rec])
