"""Pins of the oracle's SIPG matrix (Section 2, Eqs. ip / discrete / A, Section 4 penalty)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle.gll import gll_nodes, lagrange_eval
from oracle.sipg import (Mesh, assemble, assemble_1d, local_index, mass_diagonal, node_coordinates,
                         penalty, stability_threshold, weak_rhs)
from paper_1612_04796_gb300 import inputs


def kron_operator(mesh, P, factor=2.0):
    """Eq. (A) from the 1D factors, permuted to element-blocked numbering."""
    n = P + 1
    Ls, Ms = [], []
    for d in range(3):
        L, M = assemble_1d(mesh.counts[d], mesh.lengths[d], P, factor)
        Ls.append(L)
        Ms.append(np.diag(M))
    A = (np.kron(Ms[2], np.kron(Ms[1], Ls[0])) + np.kron(Ms[2], np.kron(Ls[1], Ms[0]))
         + np.kron(Ls[2], np.kron(Ms[1], Ms[0])))
    i, j, k = local_index(n)
    ex, ey, ez = mesh.element_coords()
    gx = (ex[:, None] * n + i[None, :]).ravel()
    gy = (ey[:, None] * n + j[None, :]).ravel()
    gz = (ez[:, None] * n + k[None, :]).ravel()
    perm = gx + mesh.counts[0] * n * (gy + mesh.counts[1] * n * gz)
    return A[np.ix_(perm, perm)]


@pytest.mark.parametrize("P", [1, 2, 3])
def test_symmetric_with_constant_nullspace(P):
    mesh = Mesh((1.0, 2.0, 0.5), (3, 4, 2))
    A = assemble(mesh, P)
    scale = abs(A).max()
    assert abs(A - A.T).max() <= 1e-14 * scale
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) <= 1e-13 * scale


def test_positive_semidefinite_one_dimensional_nullspace():
    A = assemble(Mesh((1, 1, 1), (3, 3, 3)), 2).toarray()
    ev = np.linalg.eigvalsh(A)
    assert abs(ev[0]) < 1e-12 * ev[-1]
    assert ev[1] > 1e-3 * ev[-1] * 1e-2


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_kronecker_form_eq_A(P):
    """The 3D element/face assembly equals Mz(x)My(x)Lx + Mz(x)Ly(x)Mx + Lz(x)My(x)Mx."""
    mesh = Mesh((1.0, 2.0, 0.5), (3, 2, 4))
    A = assemble(mesh, P).toarray()
    Ak = kron_operator(mesh, P)
    assert np.max(np.abs(A - Ak)) <= 1e-13 * np.max(np.abs(A))


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16])
def test_coercivity_threshold_is_half_of_quoted_formula(P):
    """L(mu) is PSD for mu slightly above P(P+1)/(2h) and indefinite slightly below
    (so the threshold is that value; Section 4 quotes twice it)."""
    h = 0.5
    mu0 = stability_threshold(P, h)
    assert mu0 == pytest.approx(P * (P + 1) / (2 * h))
    for fac, psd in ((1.001, True), (0.999, False)):
        L, _ = assemble_1d(6, 6 * h, P, factor=fac)  # even count: the unstable mode alternates per element
        ev = np.linalg.eigvalsh(L)
        assert (ev[0] > -1e-10 * ev[-1]) == psd
    assert penalty(P, h) == pytest.approx(P * (P + 1) / h)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_1d_generalised_eigenvalues_converge_at_order_2p(P):
    """Lowest nonzero eigenvalues of L v = lam M v on a periodic interval of
    length l are double and approach (2 pi / l)^2 with error O(h^(2P))."""
    import scipy.linalg as sla
    l = 3.0
    exact = (2 * math.pi / l) ** 2
    errs = []
    for n in (8, 16):
        L, M = assemble_1d(n, l, P)
        ev = sla.eigh(L, np.diag(M), eigvals_only=True)
        assert abs(ev[0]) < 1e-10 and ev[1] > 0
        assert ev[1] == pytest.approx(ev[2], rel=1e-9)
        errs.append(abs(ev[1] - exact) / exact)
    order = math.log2(errs[0] / errs[1])
    assert 2 * P - 0.3 < order < 2 * P + 0.5, (errs, order)


def _l2_error(P, n):
    mesh = Mesh((1, 1, 1), (n, n, n))
    A = assemble(mesh, P)
    X, Y, Z = node_coordinates(mesh, P)
    _, f = inputs.sines(X, Y, Z)
    b = weak_rhs(mesh, P, f)
    # A is SPD on the complement of the constants and 1^T b = 0: textbook CG
    u, info = spl.cg(A, b, rtol=1e-13, atol=0.0, maxiter=20000)
    assert info == 0
    xg, wg = np.polynomial.legendre.leggauss(P + 3)
    phi = lagrange_eval(gll_nodes(P), xg)
    U = u.reshape(-1, P + 1, P + 1, P + 1)
    Ug = np.einsum("ai,bj,ck,ekji->ecba", phi, phi, phi, U)
    ex, ey, ez = mesh.element_coords()
    h = mesh.h
    xq = ex[:, None] * h[0] + (xg[None, :] + 1) * h[0] / 2
    yq = ey[:, None] * h[1] + (xg[None, :] + 1) * h[1] / 2
    zq = ez[:, None] * h[2] + (xg[None, :] + 1) * h[2] / 2
    ue = (np.sin(2 * np.pi * zq)[:, :, None, None] * np.sin(2 * np.pi * yq)[:, None, :, None]
          * np.sin(2 * np.pi * xq)[:, None, None, :])
    W = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * h[0] * h[1] * h[2] / 8
    err = Ug - ue
    err = err - np.sum(W[None] * err)
    return math.sqrt(np.sum(W[None] * err ** 2))


@pytest.mark.parametrize("P,n", [(2, 4), (3, 3)])
def test_l2_convergence_order_p_plus_1(P, n):
    """Manufactured periodic solution: the L2 error decays like h^(P+1)."""
    e1, e2 = _l2_error(P, n), _l2_error(P, 2 * n)
    order = math.log2(e1 / e2)
    assert P + 1 - 0.4 < order < P + 1 + 0.6, order


def test_row_subset_assembly_matches_full():
    mesh = Mesh((1, 1, 1), (3, 4, 3))
    P = 2
    A = assemble(mesh, P)
    sel = [0, 5, 17, 35]
    As = assemble(mesh, P, row_elements=sel)
    B = (P + 1) ** 3
    rows = np.concatenate([np.arange(e * B, (e + 1) * B) for e in sel])
    assert abs(As[rows] - A[rows]).max() == 0.0
    other = np.setdiff1d(np.arange(A.shape[0]), rows)
    assert As[other].nnz == 0


def test_weak_rhs_is_compatible_and_mass_weighted():
    mesh = Mesh((2.0, 1.0, 1.0), (3, 3, 4))
    P = 3
    f = inputs.gaussian(mesh.num_elements * (P + 1) ** 3, 7)
    b = weak_rhs(mesh, P, f)
    assert abs(b.sum()) < 1e-14 * np.abs(b).sum()
    m = mass_diagonal(mesh, P)
    assert m.sum() == pytest.approx(2.0, rel=1e-13)
    # a constant rhs gives b = 0
    assert np.max(np.abs(weak_rhs(mesh, P, np.ones_like(f)))) < 1e-15
