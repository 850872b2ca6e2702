"""Pins of the learned-preconditioner oracle (oracle/learned.py)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import pytest

from oracle import learned


def _laplacian(n, shift=0.1):
    T = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    A = sp.kron(sp.identity(n), T) + sp.kron(T, sp.identity(n)) + shift * sp.identity(n * n)
    return sp.csr_matrix(A)


def test_pcg_matches_direct_solve():
    A = _laplacian(12)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(A.shape[0])
    x, k, res = learned.pcg(A, b, tol=1e-12, maxit=500)
    xd = spla.spsolve(A.tocsc(), b)
    assert res <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-10
    assert 0 < k <= A.shape[0]


def test_cg_terminates_after_distinct_eigenvalue_count():
    # Textbook Krylov fact: with k distinct eigenvalues CG terminates in <= k steps.
    d = np.repeat([1.0, 2.0, 5.0, 11.0], 25)
    A = sp.diags(d).tocsr()
    b = np.ones(len(d))
    _, k, res = learned.pcg(A, b, tol=1e-12)
    assert k <= 4 and res <= 1e-12
    # The exact inverse as preconditioner converges in one step.
    _, k1, _ = learned.pcg(A, b, apply_minv=lambda r: r / d, tol=1e-12)
    assert k1 == 1


def _small_problem(seed=1, n=7, ns=3):
    A = _laplacian(n, 0.3)
    indptr, indices = learned.lower_pattern(A)
    rng = np.random.default_rng(seed)
    vals = rng.standard_normal(len(indices)) * 0.3
    R = rng.standard_normal((A.shape[0], ns))
    X = spla.spsolve(A.tocsc(), R)
    return A, indptr, indices, vals, R, X


def test_fsai_gradient_matches_central_differences():
    A, indptr, indices, vals, R, X = _small_problem()
    loss, g = learned.fsai_loss_grad(indptr, indices, vals, R, X)
    rng = np.random.default_rng(7)
    for k in rng.choice(len(vals), 12, replace=False):
        h = 1e-6 * max(1.0, abs(vals[k]))
        vp = vals.copy(); vp[k] += h
        vm = vals.copy(); vm[k] -= h
        fd = (learned.fsai_loss_grad(indptr, indices, vp, R, X)[0] -
              learned.fsai_loss_grad(indptr, indices, vm, R, X)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])
    # The loss itself, written out for one sample.
    G = learned.fsai_matrix(indptr, indices, vals, A.shape[0])
    e0 = G @ (G.T @ R[:, 0]) - X[:, 0]
    single = learned.fsai_loss_grad(indptr, indices, vals, R[:, :1], X[:, :1])[0]
    assert single == pytest.approx(float(e0 @ e0 / (X[:, 0] @ X[:, 0])), rel=1e-12)


def test_exact_inverse_factor_has_zero_loss_and_one_pcg_step():
    # With the full lower pattern, G = chol(S^{-1}) (lower) gives G G^T = S^{-1}.
    A = _laplacian(5, 0.5).toarray()
    n = A.shape[0]
    Gd = np.linalg.cholesky(np.linalg.inv(A))
    full = sp.csr_matrix(np.tril(np.ones((n, n))))
    full.sort_indices()
    indptr, indices = full.indptr, full.indices
    vals = np.array([Gd[i, j] for i in range(n) for j in indices[indptr[i]:indptr[i + 1]]])
    rng = np.random.default_rng(3)
    R = rng.standard_normal((n, 4))
    X = np.linalg.solve(A, R)
    loss, g = learned.fsai_loss_grad(indptr, indices, vals, R, X)
    assert loss <= 1e-24 and np.abs(g).max() <= 1e-10
    G = learned.fsai_matrix(indptr, indices, vals, n)
    _, k, _ = learned.pcg(sp.csr_matrix(A), R[:, 0], apply_minv=lambda r: learned.fsai_apply(G, r), tol=1e-10)
    assert k == 1


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = learned.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # Bias correction makes m_hat = g and v_hat = g^2 at t = 1.
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_kaporin_gradient_matches_central_differences():
    A, indptr, indices, vals, R, X = _small_problem(seed=4)
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(indptr))
    vals = vals.copy()
    vals[indices == rows] = 1.0 + np.abs(vals[indices == rows])   # log needs a positive diagonal
    loss, g = learned.kaporin_loss_grad(A, indptr, indices, vals)
    rng = np.random.default_rng(9)
    for k in rng.choice(len(vals), 12, replace=False):
        h = 1e-6
        vp = vals.copy(); vp[k] += h
        vm = vals.copy(); vm[k] -= h
        fd = (learned.kaporin_loss_grad(A, indptr, indices, vp)[0] -
              learned.kaporin_loss_grad(A, indptr, indices, vm)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])
    # tr(G^T S G) written out with dense matrices.
    G = learned.fsai_matrix(indptr, indices, vals, n).toarray()
    dense = np.trace(G.T @ A.toarray() @ G) - 2 * np.sum(np.log(np.diag(G)))
    assert loss == pytest.approx(dense, rel=1e-12)


def test_kaporin_minimiser_is_the_closed_form_fsai():
    A = _laplacian(6, 0.2)
    indptr, indices = learned.lower_pattern(A)
    vc = learned.fsai_closed_form(A, indptr, indices)
    _, g = learned.kaporin_loss_grad(A, indptr, indices, vc)
    assert np.abs(g).max() <= 1e-10
    # Full lower pattern: the closed form is the lower Cholesky factor of S^{-1}.
    n = A.shape[0]
    full = sp.csr_matrix(np.tril(np.ones((n, n))))
    full.sort_indices()
    vf = learned.fsai_closed_form(A, full.indptr, full.indices)
    Gd = np.linalg.cholesky(np.linalg.inv(A.toarray()))
    assert np.allclose(learned.fsai_matrix(full.indptr, full.indices, vf, n).toarray(), Gd, atol=1e-12)
    # Adam on K approaches it.
    vt, hist = learned.train_fsai_kaporin(A, indptr, indices, epochs=3000, lr=1e-2)
    assert hist[-1] < hist[0]
    assert np.linalg.norm(vt - vc) <= 1e-3 * np.linalg.norm(vc)


def _method_pairs():
    # (r, a = S^{-1} r) from the method's own implicit solves on the 16x16-cell plate.
    from oracle import pipeline
    from paper_2310_14712_gb300 import workloads
    w = workloads.plate16()
    s = pipeline.setup(**w.kwargs())
    im = s.imex
    d = s.disc
    Ic = np.flatnonzero(d.is_c)
    S = sp.csr_matrix(d.M[Ic][:, Ic] + 0.25 * s.dt ** 2 * d.K[Ic][:, Ic])
    rhs, sol = [], []
    state = im.initial_state()
    for n in range(60):
        state = im.step(state)
        if n % 3 == 0:
            sol.append(state.a_c[Ic])
            rhs.append(S @ state.a_c[Ic])
    return S, np.array(rhs).T, np.array(sol).T


def test_learned_preconditioner_shortens_cg_on_the_methods_systems():
    # The trained FSAI against its untrained (Jacobi) start, on the right-hand
    # sides the method produces; the direct solve judges the error.
    S, R, X = _method_pairs()
    indptr, indices = learned.lower_pattern(S)
    v0 = learned.jacobi_init(indptr, indices, S)
    vals, hist = learned.train_fsai_kaporin(S, indptr, indices, epochs=600, lr=3e-2)
    assert hist[-1] < hist[0]
    G0 = learned.fsai_matrix(indptr, indices, v0, S.shape[0])
    G1 = learned.fsai_matrix(indptr, indices, vals, S.shape[0])
    k0 = k1 = 0
    for j in range(R.shape[1]):
        x0, i0, _ = learned.pcg(S, R[:, j], apply_minv=lambda r: learned.fsai_apply(G0, r), tol=1e-10)
        x1, i1, r1 = learned.pcg(S, R[:, j], apply_minv=lambda r: learned.fsai_apply(G1, r), tol=1e-10)
        k0 += i0
        k1 += i1
        assert r1 <= 1e-10
        assert np.linalg.norm(x1 - X[:, j]) <= 1e-6 * np.linalg.norm(X[:, j])
    assert k1 < 0.5 * k0


# --- learned starting guess (extrapolation weights) ---------------------------

def _quadratic_sequence(n=40, T=12, seed=3):
    rng = np.random.default_rng(seed)
    c0, c1, c2 = rng.standard_normal((3, n))
    t = np.arange(T, dtype=np.float64)
    return c0[:, None] + c1[:, None] * t + c2[:, None] * t * t     # (n, T)


def test_extrapolation_exact_on_quadratic_sequences():
    # Polynomial extrapolation through the last three values reproduces any
    # sequence quadratic in time: the loss is zero at w = (3, -3, 1), and this
    # is its unique minimiser when the three histories are independent.
    A = _quadratic_sequence()
    H, X = learned.extrapolation_samples(A, 3)
    loss, g = learned.extrapolation_loss_grad(H, X, [3.0, -3.0, 1.0])
    assert loss <= 1e-24 and np.abs(g).max() <= 1e-10
    assert np.allclose(learned.extrapolation_guess(H, [3.0, -3.0, 1.0]), X, rtol=0, atol=1e-10)
    # Written out for one sample: the loss of w = (1, 0, 0) (start from a_n).
    s = 4
    e = A[:, s + 2] - A[:, s + 3]
    l1, _ = learned.extrapolation_loss_grad(H[:, :, s:s + 1], X[:, s:s + 1], [1.0, 0.0, 0.0])
    assert l1 == pytest.approx(e @ e / (A[:, s + 3] @ A[:, s + 3]), rel=1e-13)


def test_extrapolation_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 9)).cumsum(axis=1)
    H, X = learned.extrapolation_samples(A, 3)
    w = np.array([1.7, -0.9, 0.2])
    loss, g = learned.extrapolation_loss_grad(H, X, w)
    for k in range(3):
        h = 1e-6
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd = (learned.extrapolation_loss_grad(H, X, wp)[0] - learned.extrapolation_loss_grad(H, X, wm)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_adam_learns_the_quadratic_extrapolation():
    A = _quadratic_sequence()
    H, X = learned.extrapolation_samples(A, 3)
    w, hist = learned.train_extrapolation(H, X, [1.0, 0.0, 0.0], 3000, 0.05)
    assert hist[-1] < 1e-12 * hist[0]
    assert np.allclose(w, [3.0, -3.0, 1.0], atol=1e-5), w


def test_learned_guess_cuts_cg_iterations_on_the_methods_own_solves():
    # The plate's accelerations a^c_n from the oracle's own run: weights
    # learned on steps 100..160 start the solves of steps 170..190 closer to
    # their solutions than a_n does, and CG needs fewer iterations there.
    from oracle import pipeline
    from paper_2310_14712_gb300 import workloads
    w_ = workloads.plate16(steps=200)
    s = pipeline.setup(**w_.kwargs())
    Ic = s.imex.Ic
    st = s.imex.initial_state()
    acc, rhs = [], []
    for n in range(190):
        st = s.imex.step(st)
        acc.append(st.a_c[Ic].copy())
    A = np.stack(acc, axis=1)
    H, X = learned.extrapolation_samples(A[:, 100:161], 3)
    w, hist = learned.train_extrapolation(H, X, [1.0, 0.0, 0.0], 2000, 0.01)
    assert hist[-1] < 0.1 * hist[0]
    d = s.disc
    S = sp.csr_matrix(d.M[Ic][:, Ic] + 0.25 * s.dt ** 2 * d.K[Ic][:, Ic])
    its_plain, its_learned = 0, 0
    for n in range(170, 189):
        b = S @ A[:, n + 1]
        x0p = A[:, n]
        x0l = learned.extrapolation_guess(A[:, [n, n - 1, n - 2]].T, w)
        _, kp, _ = learned.pcg(S, b, x0=x0p, apply_minv=lambda r: r / S.diagonal(), tol=1e-10, maxit=5000)
        _, kl, _ = learned.pcg(S, b, x0=x0l, apply_minv=lambda r: r / S.diagonal(), tol=1e-10, maxit=5000)
        its_plain += kp
        its_learned += kl
    assert its_learned < 0.9 * its_plain, (its_learned, its_plain)
