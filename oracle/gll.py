"""Gauss-Legendre-Lobatto nodal basis on the reference interval [-1, 1].

Section 2 (Eq. u_h): the 1D base functions phi_i are the Lagrange polynomials
to the P+1 GLL points; the same points serve as quadrature rule ("applying ...
GLL quadrature").

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def _legendre_coeffs(P):
    c = np.zeros(P + 1)
    c[P] = 1.0
    return c


def gll_nodes(P):
    """The P+1 GLL points: -1, +1 and the P-1 roots of the derivative of the
    Legendre polynomial L_P, in increasing order."""
    if P < 1:
        raise ValueError("P must be >= 1")
    if P == 1:
        return np.array([-1.0, 1.0])
    dc = npleg.legder(_legendre_coeffs(P))
    roots = np.sort(npleg.legroots(dc).real)
    d2c = npleg.legder(dc)
    for _ in range(3):  # Newton polish of L_P'(x) = 0
        roots = roots - npleg.legval(roots, dc) / npleg.legval(roots, d2c)
    return np.concatenate([[-1.0], roots, [1.0]])


def gll_weights(P):
    """GLL quadrature weights w_i = 2 / (P (P+1) L_P(x_i)^2)."""
    x = gll_nodes(P)
    lp = npleg.legval(x, _legendre_coeffs(P))
    return 2.0 / (P * (P + 1) * lp ** 2)


def lagrange_eval(nodes, x):
    """Phi[q, j] = phi_j(x_q) for the Lagrange basis on ``nodes``, by the product
    formula phi_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    phi = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                phi[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return phi


def diff_matrix(nodes):
    """D[q, j] = phi_j'(x_q), by differentiating the product formula:
    off the diagonal, phi_j'(x_q) = prod_{m != j, q} (x_q - x_m) / prod_{m != j} (x_j - x_m);
    on it, phi_q'(x_q) = sum_{m != q} 1 / (x_q - x_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    D = np.zeros((n, n))
    for q in range(n):
        for j in range(n):
            if q == j:
                D[q, q] = sum(1.0 / (nodes[q] - nodes[m]) for m in range(n) if m != q)
            else:
                num = 1.0
                for m in range(n):
                    if m != j and m != q:
                        num *= nodes[q] - nodes[m]
                den = 1.0
                for m in range(n):
                    if m != j:
                        den *= nodes[j] - nodes[m]
                D[q, j] = num / den
    return D
