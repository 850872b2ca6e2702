"""Learned preconditioner for the implicit solve S a = r of the Newmark IMEX
step, and the preconditioned conjugate gradient method that uses it (oracle,
test infrastructure: imported only by the tests, the smoke check and the
bench's CPU leg).

The paper solves S a = r (Fig. TrapCDMIMEX, "Acceleration calculation") with
a factorisation computed once.  This module is the CPU definition of the
alternative: conjugate gradients with a preconditioner learned from pairs
(r, a = S^{-1} r) that the method itself produces.

  * pcg: preconditioned conjugate gradients (Saad, Iterative Methods for
    Sparse Linear Systems, 2nd ed., Algorithm 9.1), stopping when
    ||r_k|| <= tol ||b||.
  * The preconditioner is a factorised sparse approximate inverse
    M^{-1} = G G^T with G lower triangular on a fixed sparsity pattern
    (Kolotilina and Yeremin's FSAI form); it is symmetric positive definite
    whenever G has a nonzero diagonal, so CG stays valid.  G is learned, not
    computed from S: the loss over sample pairs (r_s, x_s) is
        L(G) = sum_s ||G G^T r_s - x_s||^2 / ||x_s||^2,
    and its gradient on the pattern follows from the chain rule through
    z = G^T r, y = G z (fsai_loss_grad).
  * adam_step: one step of Adam (Kingma and Ba, 2015, Algorithm 1).
  * The training objective actually used: Kaporin's condition-number
    functional for the factorised form, K(G) = tr(G^T S G) - 2 sum_i log G_ii
    (log of the K-condition number of G^T S G up to constants; convex on
    the pattern).  Its stationary point is, column by column,
    S_QQ g_j = e_j / G_jj on the rows Q of column j of the pattern, i.e. the
    classical FSAI of the pattern (fsai_closed_form).  The data-fit loss
    above is kept as the check on the method's own pairs: fitting it alone
    lengthened CG on held-out right-hand sides.

  * The starting guess of each solve is learned from the method's own
    solutions: x0 = sum_k w_k a_{n-k} (k < 3, a_n the accelerations of the
    last solves; PCG otherwise starts from a_n), with the weights w fitted by
    Adam to the loss over consecutive solutions
        E(w) = sum_s ||sum_k w_k a_{s-k} - a_{s+1}||^2 / ||a_{s+1}||^2
    (extrapolation_loss_grad).  Polynomial extrapolation through the last
    three values, w = (3, -3, 1), is exact for accelerations quadratic in
    time; the learned weights adapt to the wave content of the run.

Pins (tests/test_oracle_learned.py): PCG against a direct solve and its
iteration bound on a diagonal system; both gradients against central finite
differences and the losses written out densely; the data-fit loss at the
exact inverse factor (zero, and PCG converging in one iteration); the
Kaporin minimiser against the column-wise closed form (and, on the full
lower pattern, the Cholesky factor of S^{-1}); Adam's first step in closed
form; training on the method's own systems halving CG iterations against
the untrained (Jacobi) start, the direct solve judging the error; the
extrapolation loss zero at w = (3, -3, 1) on any sequence quadratic in time,
its gradient against central differences, Adam converging to those weights
on such a sequence, and the learned guess cutting CG iterations on later
solves of the method's own run.
"""
import numpy as np
import scipy.sparse as sp


def lower_pattern(S):
    """Sparsity pattern of the lower triangle of S (diagonal included), CSR."""
    L = sp.tril(sp.csr_matrix(S), format="csr")
    L.sort_indices()
    return L.indptr.copy(), L.indices.copy()


def fsai_matrix(indptr, indices, vals, n):
    return sp.csr_matrix((np.asarray(vals, dtype=np.float64), indices, indptr), shape=(n, n))


def fsai_apply(G, r):
    """z = G (G^T r)."""
    return G @ (G.T @ r)


def fsai_loss_grad(indptr, indices, vals, R, X):
    """Loss sum_s ||G G^T r_s - x_s||^2 / ||x_s||^2 and its gradient on the
    pattern.  R, X: (n, ns) sample matrices (columns are samples).

    With z = G^T r, y = G z, e = y - x and weight w = 1 / ||x||^2:
      dL/dy = 2 w e;  y = G z gives dL/dG_ij += (2 w e)_i z_j and
      dL/dz = G^T (2 w e);  z = G^T r gives dL/dG_ij += r_i (dL/dz)_j."""
    n = len(indptr) - 1
    G = fsai_matrix(indptr, indices, vals, n)
    R = np.asarray(R, dtype=np.float64).reshape(n, -1)
    X = np.asarray(X, dtype=np.float64).reshape(n, -1)
    w = 1.0 / np.sum(X * X, axis=0)
    Z = G.T @ R
    E = G @ Z - X
    loss = float(np.sum(w * np.sum(E * E, axis=0)))
    D = 2.0 * E * w              # dL/dY
    Q = G.T @ D                  # dL/dZ
    rows = np.repeat(np.arange(n), np.diff(indptr))
    grad = np.sum(D[rows] * Z[indices] + R[rows] * Q[indices], axis=1)
    return loss, grad


def adam_step(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new params, m, v."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def pcg(A, b, x0=None, apply_minv=None, tol=1e-10, maxit=1000):
    """Preconditioned CG (Algorithm 9.1 of Saad).  Returns x, iterations, and
    the relative residual ||b - A x|| / ||b|| it stopped at."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    minv = (lambda r: r) if apply_minv is None else apply_minv
    r = b - A @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    if np.linalg.norm(r) <= tol * nb:
        return x, 0, float(np.linalg.norm(r) / nb)
    z = minv(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        res = np.linalg.norm(r) / nb
        if res <= tol:
            return x, k, float(res)
        z = minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, float(np.linalg.norm(r) / nb)


def kaporin_loss_grad(S, indptr, indices, vals):
    """K(G) = tr(G^T S G) - 2 sum_i log G_ii and its gradient on the pattern:
    tr(G^T S G) = sum over the pattern of G_ij (S G)_ij, gradient 2 (S G)_ij
    - 2 delta_ij / G_ii."""
    n = len(indptr) - 1
    G = fsai_matrix(indptr, indices, vals, n)
    SG = sp.csr_matrix(S) @ G
    rows = np.repeat(np.arange(n), np.diff(indptr))
    sg = np.asarray(SG[rows, indices]).ravel()
    diag = indices == rows
    loss = float(np.dot(vals, sg) - 2.0 * np.sum(np.log(vals[diag])))
    grad = 2.0 * sg
    grad[diag] -= 2.0 / vals[diag]
    return loss, grad


def fsai_closed_form(S, indptr, indices):
    """Minimiser of K on the pattern, column by column: with Q the rows of
    column j, solve S_QQ y = e_j and set G_Qj = y / sqrt(y_j)."""
    n = len(indptr) - 1
    S = sp.csr_matrix(S)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    vals = np.zeros(len(indices))
    for j in range(n):
        ks = np.flatnonzero(indices == j)
        Q = rows[ks]
        y = np.linalg.solve(S[Q][:, Q].toarray(), (Q == j).astype(np.float64))
        vals[ks] = y / np.sqrt(y[Q == j][0])
    return vals


def train_fsai_kaporin(S, indptr, indices, epochs, lr, diag_floor=1e-3):
    """Adam on K from the Jacobi start, in row-scaled units theta = G_ij
    sqrt(S_ii) (so theta_ii = 1 at the start); the diagonal is kept at or
    above diag_floor so that G G^T stays positive definite.  Returns the
    values and the loss history."""
    n = len(indptr) - 1
    rows = np.repeat(np.arange(n), np.diff(indptr))
    scale = 1.0 / np.sqrt(np.asarray(sp.csr_matrix(S).diagonal(), dtype=np.float64))[rows]
    diag = indices == rows
    th = jacobi_init(indptr, indices, S) / scale
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    hist = []
    for t in range(1, epochs + 1):
        loss, g = kaporin_loss_grad(S, indptr, indices, th * scale)
        hist.append(loss)
        th, m, v = adam_step(th, g * scale, m, v, t, lr)
        th[diag] = np.maximum(th[diag], diag_floor)
    return th * scale, hist


def jacobi_init(indptr, indices, S):
    """G = diag(S)^{-1/2} on the pattern (the untrained start: M^{-1} = D^{-1})."""
    d = np.asarray(sp.csr_matrix(S).diagonal(), dtype=np.float64)
    n = len(indptr) - 1
    vals = np.zeros(len(indices))
    for i in range(n):
        for k in range(indptr[i], indptr[i + 1]):
            if indices[k] == i:
                vals[k] = 1.0 / np.sqrt(d[i])
    return vals


def extrapolation_guess(H, w):
    """x0 = sum_k w_k H[k]; H: (K, n, ...) histories, H[k] = a_{n-k}."""
    H = np.asarray(H, dtype=np.float64)
    return np.tensordot(np.asarray(w, dtype=np.float64), H, axes=(0, 0))


def extrapolation_loss_grad(H, X, w):
    """E(w) = sum_s ||sum_k w_k H[k][:, s] - X[:, s]||^2 / ||X[:, s]||^2 and its
    gradient dE/dw_k = sum_s 2 (e_s . H[k][:, s]) / ||X[:, s]||^2, e_s the
    residual of sample s.  H: (K, n, ns), X: (n, ns)."""
    H = np.asarray(H, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    wt = 1.0 / np.sum(X * X, axis=0)
    E = extrapolation_guess(H, w) - X
    loss = float(np.sum(wt * np.sum(E * E, axis=0)))
    grad = np.array([float(np.sum(2.0 * wt * np.sum(E * H[k], axis=0))) for k in range(H.shape[0])])
    return loss, grad


def extrapolation_samples(A, K=3):
    """Histories and targets from a sequence of solutions A (n, T): sample s
    (K-1 <= s < T-1) has H[k][:, s] = A[:, s-k] and target A[:, s+1]."""
    A = np.asarray(A, dtype=np.float64)
    T = A.shape[1]
    s = np.arange(K - 1, T - 1)
    H = np.stack([A[:, s - k] for k in range(K)])
    return H, A[:, s + 1]


def train_extrapolation(H, X, w0, epochs, lr):
    """Full-batch Adam on E from w0; returns w and the loss history."""
    w = np.array(w0, dtype=np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    hist = []
    for t in range(1, epochs + 1):
        loss, g = extrapolation_loss_grad(H, X, w)
        hist.append(loss)
        w, m, v = adam_step(w, g, m, v, t, lr)
    return w, hist
