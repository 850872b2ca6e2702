"""1D spectral basis of the spectral cell method (oracle, test infrastructure).

Follows Sec. "Spatial discretization": Lagrange polynomials of degree p on the
p+1 Gauss-Lobatto-Legendre (GLL) points (Eq. Lagrange and the GLL point
definition), and Gauss-Legendre (GL) quadrature, which the paper uses for all
stiffness and load integrals and for the mass of cut cells.

The paper defines the interior GLL points as "roots of Lobatto polynomials of
order p-1"; that is the same point set as the roots of P_p', the derivative of
the Legendre polynomial of degree p, which is what is computed here.

Pins (tests/test_oracle_basis.py): textbook GLL tables for p = 2 and 4, weights
summing to 2, exactness of GLL quadrature up to degree 2p-1 and of GL up to
2n-1, the Kronecker-delta and partition-of-unity properties of the basis, and
the single-cell eigenfrequencies the paper prints (Fig. fillRatioHZ data).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_points(p):
    """GLL points and weights of order p (p+1 points, ascending) on [-1, 1].

    Points: -1, the p-1 roots of P_p', +1.  Weights: w_j = 2 / (p (p+1) P_p(xi_j)^2).
    """
    if p < 1:
        raise ValueError("p >= 1 required")
    cp = np.zeros(p + 1)
    cp[p] = 1.0                       # Legendre series of P_p
    inner = np.zeros(0)
    if p >= 2:
        r = npleg.legroots(npleg.legder(cp))
        if np.iscomplexobj(r):
            if np.max(np.abs(r.imag)) > 1e-12:
                raise ValueError("complex GLL roots")
            r = r.real
        inner = np.sort(r)
    x = np.concatenate(([-1.0], inner, [1.0]))
    w = 2.0 / (p * (p + 1) * npleg.legval(x, cp) ** 2)
    return x, w


def gauss_points(n):
    """n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    x, w = npleg.leggauss(n)
    return x, w


def lagrange(nodes, xi):
    """Values N_i(xi_q) of the Lagrange polynomials on `nodes`; shape (len(xi), len(nodes))."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(xi), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                out[:, i] *= (xi - nodes[j]) / (nodes[i] - nodes[j])
    return out


def lagrange_deriv(nodes, xi):
    """Derivatives N_i'(xi_q) by the product rule; shape (len(xi), len(nodes))."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    n = len(nodes)
    out = np.zeros((len(xi), n))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.full(len(xi), 1.0 / (nodes[i] - nodes[k]))
            for j in range(n):
                if j != i and j != k:
                    term *= (xi - nodes[j]) / (nodes[i] - nodes[j])
            out[:, i] += term
    return out
