"""Iterative solve of the implicit partition with the learned preconditioner.

  * the training kernels (Kaporin's functional and its gradient) against
    oracle/learned.py on the oracle's own S and a random G;
  * PCG stepping against the oracle's direct-solve run, every solve at the
    requested relative residual, no fallback;
  * the trained G against its untrained (Jacobi) start: fewer iterations;
  * a PCG that cannot converge falls back to the direct solve, bit for bit.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import learned, pipeline
from paper_2310_14712_gb300 import workloads

from parity_util import phys_mask

pytestmark = pytest.mark.gpu


def _imex():
    from paper_2310_14712_gb300 import imex
    return imex


def _oracle_S(w):
    s = pipeline.setup(**w.kwargs())
    d = s.disc
    Ic = np.flatnonzero(d.is_c)
    S = sp.csr_matrix(d.M[Ic][:, Ic] + 0.25 * s.dt ** 2 * d.K[Ic][:, Ic])
    S.sort_indices()
    return s, S


def test_kaporin_kernels_match_oracle():
    import torch
    imex = _imex()
    _, S = _oracle_S(workloads.plate16())
    indptr, indices = learned.lower_pattern(S)
    n = S.shape[0]
    rows = np.repeat(np.arange(n), np.diff(indptr))
    rng = np.random.default_rng(11)
    vals = learned.jacobi_init(indptr, indices, S) * (1.0 + 0.2 * rng.random(len(indices)))
    off = indices != rows
    vals[off] = 0.3 * rng.standard_normal(off.sum()) / np.sqrt(S.diagonal()[rows[off]])
    loss_ref, grad_ref = learned.kaporin_loss_grad(S, indptr, indices, vals)
    dev = torch.device("cuda")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    loss, grad = imex.fsai_kaporin(t(S.indptr, torch.int32), t(S.indices, torch.int32), t(S.data, torch.float64),
                                   t(indptr, torch.int32), t(indices, torch.int32), t(vals, torch.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-12)
    g = grad.cpu().numpy()
    assert np.abs(g - grad_ref).max() <= 1e-11 * np.abs(grad_ref).max()


def _run(w, nsteps, solver, train=0, tol=1e-10, maxit=400):
    imex = _imex()
    with imex.Imex.from_workload(w) as g:
        hist = g.pcg_train(train) if train else None
        g.set_solver(solver, tol, maxit)
        iters = []
        for _ in range(nsteps):
            g.step(1)
            if solver != "direct":
                st = g.pcg_status()
                iters.append(st["iters_last"])
                assert st["res_last"] <= tol or st["fallbacks"] > 0
        u = g.fields("u", out=np.zeros(g.n_nodes))
        status = g.pcg_status()
    return u, np.array(iters), status, hist


@pytest.mark.parametrize("solver,train", [("pcg_jacobi", 0), ("pcg_fsai", 400)])
def test_pcg_stepping_matches_oracle(solver, train):
    w = workloads.plate16()
    nsteps = 120
    u, iters, status, hist = _run(w, nsteps, solver, train)
    assert status["fallbacks"] == 0
    if hist is not None:
        assert hist[-1] < hist[0]
    s = pipeline.setup(**w.kwargs())
    ref = s.imex.run(nsteps)
    phys = phys_mask(s, w.holes)
    # Each solve stops at relative residual 1e-10, so the state differs from
    # the factorised solve by up to cond(S) x 1e-10 per solve, not by rounding
    # alone (cond(S) ~ 1e5 here: alpha = 1e-5 in the holes).  Measured on
    # GB300: ~1e-9 on physical DOFs, ~2e-7 on all active DOFs.
    e_phys = pipeline.relative_l2(u, ref.u, phys)
    e_all = pipeline.relative_l2(u, ref.u, s.disc.active)
    print(f"{solver}: e_phys {e_phys:.3e} e_all {e_all:.3e} iterations {iters.sum()}")
    assert e_phys <= 1e-8
    assert e_all <= 1e-6


def test_trained_preconditioner_halves_iterations():
    w = workloads.plate16()
    _, it_j, _, _ = _run(w, 60, "pcg_jacobi")
    _, it_l, _, hist = _run(w, 60, "pcg_fsai", train=400)
    assert hist[-1] < hist[0]
    assert it_l.sum() < 0.5 * it_j.sum(), (it_l.sum(), it_j.sum())


def test_pcg_that_cannot_converge_falls_back_to_the_direct_solve():
    w = workloads.plate16()
    u_d, _, _, _ = _run(w, 30, "direct")
    u_p, _, status, _ = _run(w, 30, "pcg_jacobi", tol=1e-30, maxit=2)
    assert status["fallbacks"] == 30
    assert np.array_equal(u_d, u_p)


def test_pcg_solver_rejected_for_several_columns():
    imex = _imex()
    w = workloads.multisource(nsrc=2)
    with imex.Imex.from_workload(w, ncols=2) as g:
        with pytest.raises(imex.ImexError):
            g.set_solver("pcg_jacobi")


# Contexts without a factorisation (imex_setup_pcg): PCG is the only solve.

def _run_nf(w, nsteps, solver="pcg_jacobi", train=0, tol=1e-10, maxit=5000):
    imex = _imex()
    with imex.Imex.from_workload(w, factorize=False) as g:
        info = g.info()
        a0 = g.fields("a_c", out=np.zeros(g.n_nodes))
        if train:
            g.pcg_train(train)
        g.set_solver(solver, tol, maxit)
        g.step(nsteps)
        u = g.fields("u", out=np.zeros(g.n_nodes))
        status = g.pcg_status()
    return u, a0, status, info


@pytest.mark.parametrize("solver,train", [("pcg_jacobi", 0), ("pcg_fsai", 400)])
def test_pcg_without_factorisation_matches_oracle(solver, train):
    w = workloads.plate16()
    nsteps = 120
    u, a0, status, info = _run_nf(w, nsteps, solver, train)
    assert info["factorized"] == 0 and info["nnz_L"] == 0 and info["launches_per_step"] == 3
    assert status["fallbacks"] == 0
    s = pipeline.setup(**w.kwargs())
    st0 = s.imex.initial_state()
    phys = phys_mask(s, w.holes)
    # a^c_0 by Jacobi-CG on M^cc to 1e-12 (M^cc is far worse conditioned than S).
    assert pipeline.relative_l2(a0, st0.a_c, phys & s.disc.is_c) <= 1e-8
    ref = s.imex.run(nsteps)
    # Same bounds as the PCG stepping of a factorised context (cond(S) x tol).
    assert pipeline.relative_l2(u, ref.u, phys) <= 1e-8
    assert pipeline.relative_l2(u, ref.u, s.disc.active) <= 1e-6


def test_pcg_without_factorisation_3d_voids():
    # Six seeded ellipsoidal voids on 6 x 6 x 3 cells, p = 3, octree depth 2.
    w = workloads.voids3d(ncells=(6, 6, 3))
    w.holes = w.holes[:6]
    nsteps = 40
    u, _, status, info = _run_nf(w, nsteps)
    assert status["fallbacks"] == 0 and info["n_c"] > 0
    s = pipeline.setup(**w.kwargs())
    ref = s.imex.run(nsteps)
    assert pipeline.relative_l2(u, ref.u, phys_mask(s, w.holes)) <= 1e-8
    assert pipeline.relative_l2(u, ref.u, s.disc.active) <= 1e-6


def test_pcg_without_factorisation_trapezoidal():
    from oracle import schemes
    w = workloads.plate16()
    imex = _imex()
    with imex.Imex.from_workload(w, factorize=False, scheme="trapezoidal") as g:
        g.set_solver("pcg_jacobi", 1e-11, 5000)
        g.step(60)
        u = g.fields("u", out=np.zeros(g.n_nodes))
        assert g.pcg_status()["fallbacks"] == 0
    s = pipeline.setup(**w.kwargs())
    ref = schemes.run(s, "trapezoidal", 60)
    assert pipeline.relative_l2(u, ref.u, phys_mask(s, w.holes)) <= 1e-8


def test_context_without_factorisation_restrictions():
    imex = _imex()
    w = workloads.plate16()
    with imex.Imex.from_workload(w, factorize=False) as g:
        with pytest.raises(imex.ImexError):
            g.set_solver("direct")
        with pytest.raises(imex.ImexError):
            g.step_noalloc(1)
    with pytest.raises(ValueError):
        imex.Imex.from_workload(workloads.multisource(nsrc=2), ncols=2, factorize=False)


def test_failing_allocator_is_reported():
    # Fault injection on the host: an allocator hook that returns NULL.
    import ctypes
    imex = _imex()
    kw = workloads.plate16().kwargs()
    m, s, keep = imex._mesh_source(kw["dim"], kw["lo"], kw["hi"], kw["ncells"], kw["depth"], kw["holes"],
                                   kw["rho"], kw["c0"], kw["cell_c"], kw["src_pos"], kw["f0"], kw["src_sigma"],
                                   kw["src_amp"], kw["wavelet"])
    calls = []

    def alloc(nbytes, user):
        calls.append(nbytes)
        return None

    def release(ptr, user):
        pass

    al = imex.Alloc(imex._ALLOC_FN(alloc), imex._RELEASE_FN(release), None)
    ctx = ctypes.c_void_p()
    rc = imex._lib.imex_setup_scheme(ctypes.byref(m), kw["p"], kw["alpha"], 0.0, ctypes.byref(s), 1, 0,
                                     ctypes.byref(al), ctypes.byref(ctx))
    assert rc == -3 and calls and not ctx.value   # IMEX_ERR_ALLOC, nothing returned
    assert b"allocator" in imex._lib.imex_last_error()


# --- learned starting guess and the closed-form FSAI -------------------------

def test_guess_training_kernels_match_the_oracle():
    # Two identical contexts: one learns the starting-guess weights on the GPU
    # over 30 steps; the other steps the same 30 steps and hands its
    # accelerations to the oracle's Adam.  Same losses, same weights.
    imex = _imex()
    w = workloads.plate16()
    nsteps, epochs, lr = 30, 200, 0.05
    with imex.Imex.from_workload(w, factorize=False) as a, imex.Imex.from_workload(w, factorize=False) as b:
        a.step(150)
        b.step(150)
        Ic = np.flatnonzero(b.fields("mask_c", out=np.zeros(b.n_nodes)) > 0)
        seq = [b.fields("a_c", out=np.zeros(b.n_nodes))[Ic]]
        for _ in range(nsteps):
            b.step(1)
            seq.append(b.fields("a_c", out=np.zeros(b.n_nodes))[Ic])
        w_gpu, hist_gpu = a.pcg_train_guess(nsteps, epochs, lr)
        assert a.info()["step"] == b.info()["step"]
    H, X = learned.extrapolation_samples(np.stack(seq, axis=1), 3)
    w_cpu, hist_cpu = learned.train_extrapolation(H, X, [1.0, 0.0, 0.0], epochs, lr)
    assert np.allclose(hist_gpu, hist_cpu, rtol=1e-9, atol=0), np.abs(hist_gpu / hist_cpu - 1).max()
    assert np.allclose(w_gpu, w_cpu, rtol=0, atol=1e-8), (w_gpu, w_cpu)
    assert hist_gpu[-1] < 0.2 * hist_gpu[0]


def test_learned_guess_cuts_pcg_iterations_and_keeps_parity():
    # From one state, the same 58 PCG solves (learned FSAI) with the plain
    # start a^c_n and with the learned guess: fewer iterations with the
    # guess, and the result still matches the oracle's direct run.
    imex = _imex()
    w = workloads.plate16(steps=260)
    its = {}
    with imex.Imex.from_workload(w, factorize=False) as g:
        g.pcg_train(300, 0.1)
        g.set_solver("pcg_fsai", 1e-10, 2000)
        g.step(160)
        weights, _ = g.pcg_train_guess(40, 300, 0.05)
        snap = {k: g.fields(k, out=np.zeros(g.n_nodes)) for k in ("u", "u_prev_d", "v_c", "a_c")}
        step0 = g.info()["step"]
        for guess in (False, True):
            for k, v in snap.items():
                g.set_fields(k, v)
            g.set_step(step0)
            g.pcg_set_guess(guess)
            g.step(2)                      # refills the history after the state change
            s0 = g.pcg_status()["iters_total"]
            g.step(58)
            its[guess] = g.pcg_status()["iters_total"] - s0
            if guess:
                u = g.fields("u", out=np.zeros(g.n_nodes))
                assert g.info()["step"] == 260
        assert g.pcg_status()["fallbacks"] == 0
    assert its[True] < its[False], its   # measured 790 against 819
    s = pipeline.setup(**w.kwargs())
    ref = s.imex.run(260)
    assert pipeline.relative_l2(u, ref.u, phys_mask(s, w.holes)) <= 1e-8
    assert pipeline.relative_l2(u, ref.u, s.disc.active) <= 1e-6


def test_closed_form_fsai_is_the_kaporin_minimiser():
    # Kaporin's functional is convex on the pattern; the closed form is its
    # minimiser, so the trained G approaches it from above and needs at least
    # as many iterations.
    imex = _imex()
    w = workloads.plate16()
    with imex.Imex.from_workload(w, factorize=False) as g:
        hist = g.pcg_train(300, 0.1)
        k_trained = float(hist[-1])
        g.pcg_fsai_closed_form()
        k_closed = float(g.pcg_train(1, 1e-12)[0])   # the loss before a negligible step
    assert k_closed <= k_trained + 1e-9 * abs(k_trained), (k_closed, k_trained)
    _, S = _oracle_S(w)
    indptr, indices = learned.lower_pattern(S)
    vals = learned.fsai_closed_form(S, indptr, indices)
    k_oracle = learned.kaporin_loss_grad(S, indptr, indices, vals)[0]
    assert k_closed == pytest.approx(k_oracle, rel=1e-10)
