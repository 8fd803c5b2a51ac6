"""Oracle pins of the "max" overlap of the anisotropic study (Section 4.2,
Table 2): delta_O,i = min(max_j 0.08 dx_j, dx_i), a different N_O per
direction, strips that may cover the whole neighbour element, and weights
normalised over the (up to three) subdomains that cover a node."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.multigrid import Hierarchy, max_overlap_widths, solve_mgcg
from oracle.schwarz import (SchwarzSmoother, layers_from_width, max_width_layers, normalised_subdomain_1d,
                            subdomain_1d, subdomain_indices)
from oracle.sipg import Mesh, assemble, assemble_1d
from paper_1612_04796_gb300 import inputs


def study_mesh(ar, counts=(8, 8, 8)):
    """The Table 2 domain (0, 2 pi AR) x (0, 2 pi ceil(AR/2)) x (0, 2 pi)."""
    return Mesh((2 * math.pi * ar, 2 * math.pi * math.ceil(ar / 2), 2 * math.pi), counts)


@pytest.mark.parametrize("ar,expect", [(1, (0.16, 0.16, 0.16)), (8, (0.16, 0.32, 1.28)),
                                       (12, (0.16, 0.32, 1.92)), (48, (0.16, 0.32, 2.0))])
def test_max_widths_closed_form(ar, expect):
    """On an n^3 tessellation dx : dy : dz = AR : ceil(AR/2) : 1, so the
    reference half-widths 2 min(0.08 dx, dx_i) / dx_i are 0.16, 0.16 AR /
    ceil(AR/2) and min(0.16 AR, 2)."""
    np.testing.assert_allclose(max_overlap_widths(study_mesh(ar), 0.08), expect, rtol=1e-14)


def test_max_width_layers_limits():
    """A strip of half-width 2 holds the whole neighbour element; below half an
    element the count agrees with the relative-overlap rule."""
    for P in (2, 4, 8, 16, 32):
        assert max_width_layers(P, 2.0) == P + 1
        for rel in (0.0, 0.08, 0.25, 0.5):
            assert max_width_layers(P, 2 * rel) == layers_from_width(P, rel)


@pytest.mark.parametrize("P", [2, 4, 8])
@pytest.mark.parametrize("delta", [0.16, 0.5, 1.0])
@pytest.mark.parametrize("profile", ["quintic", "linear", "quintic_halves", "quintic_normalised"])
def test_normalisation_is_identity_up_to_half_element(P, delta, profile):
    n_o = max_width_layers(P, delta)
    de, ii, w = subdomain_1d(P, n_o, delta, profile)
    de2, ii2, w2 = normalised_subdomain_1d(P, n_o, delta, profile)
    assert np.array_equal(de, de2) and np.array_equal(ii, ii2)
    assert np.array_equal(w, w2)


@pytest.mark.parametrize("P", [2, 4, 8])
@pytest.mark.parametrize("ar", [8, 48])
@pytest.mark.parametrize("profile", ["quintic", "linear", "quintic_halves", "quintic_normalised"])
def test_partition_of_unity_max_overlap(P, ar, profile):
    """sum_s R_s^T W_s R_s 1 = 1 with per-direction strips up to a whole element
    (the weighted corrections still average, Eq. correction:global)."""
    mesh = study_mesh(ar, (4, 4, 5))
    deltas = max_overlap_widths(mesh, 0.08)
    n_os = tuple(max_width_layers(P, d) for d in deltas)
    idx, W = subdomain_indices(mesh, P, n_os, deltas, profile)
    assert idx.shape[1] == np.prod([P + 1 + 2 * k for k in n_os])
    N = mesh.num_elements * (P + 1) ** 3
    s = np.bincount(idx.ravel(), weights=np.broadcast_to(W, idx.shape).ravel(), minlength=N)
    np.testing.assert_allclose(s, 1.0, atol=1e-14)


@pytest.mark.parametrize("P,n_os", [(2, (1, 2, 3)), (4, (5, 1, 2)), (4, (1, 3, 5))])
def test_direct_subdomain_inverse_non_cubic(P, n_os):
    """A_ss^{-1} = (Sz (x) Sy (x) Sx)(Lambda sum)^{-1}(...)^T for subdomains of
    different width per direction (Section 3.1): pins the index layout
    a + m_x (b + m_y c) of non-cubic subdomains, including strips that are
    whole neighbour elements (N_O = P + 1)."""
    mesh = Mesh((3.0, 1.5, 0.7), (4, 4, 5))
    A = assemble(mesh, P)
    deltas = tuple(min(2.0, 2.0 * k / (P + 1)) for k in n_os)
    sm = SchwarzSmoother(A, mesh, P, n_os, deltas)
    n = P + 1
    SL = []
    for d in range(3):
        L, M = assemble_1d(mesh.counts[d], mesh.lengths[d], P)
        idx = np.arange(n - n_os[d], 2 * n + n_os[d])
        lam, S = sla.eigh(L[np.ix_(idx, idx)], np.diag(M[idx]))
        SL.append((S, lam))
    (Sx, lx), (Sy, ly), (Sz, lz) = SL
    mx, my, mz = len(lx), len(ly), len(lz)
    rs = inputs.gaussian(mx * my * mz, 3)
    R = rs.reshape(mz, my, mx)
    V = np.einsum("ap,cba->cbp", Sx, R)
    V = np.einsum("bq,cbp->cqp", Sy, V)
    V = np.einsum("cr,cqp->rqp", Sz, V)
    V = V / (lz[:, None, None] + ly[None, :, None] + lx[None, None, :])
    U = np.einsum("cr,rqp->cqp", Sz, V)
    U = np.einsum("bq,cqp->cbp", Sy, U)
    U = np.einsum("ap,cbp->cba", Sx, U)
    direct = sm.local_solve(rs[:, None])[:, 0]
    np.testing.assert_allclose(direct, U.ravel(), rtol=0, atol=1e-11 * np.abs(U).max())


def _mgcg_iterations(mesh, P, **kw):
    H = Hierarchy(mesh, P, **kw)
    f = inputs.gaussian(H.levels[-1].N, 2)
    f -= f.mean()
    _, its, _ = solve_mgcg(H, f, tol=1e-10, maxit=200, growth=3)
    return its, H


def test_max_overlap_is_more_robust_than_relative():
    """Section 4.2: with the variable V-cycle, an overlap proportional to the
    largest element side ("0.08 max") converges much faster than the relative
    one ("0.08 rel") at large aspect ratios; at AR = 1 the two are the same
    method."""
    its_rel1, _ = _mgcg_iterations(study_mesh(1, (4, 4, 4)), 4, delta_rel=0.08)
    its_max1, _ = _mgcg_iterations(study_mesh(1, (4, 4, 4)), 4, max_frac=0.08)
    assert its_rel1 == its_max1
    its_rel, _ = _mgcg_iterations(study_mesh(16, (4, 4, 4)), 4, delta_rel=0.08)
    its_max, H = _mgcg_iterations(study_mesh(16, (4, 4, 4)), 4, max_frac=0.08)
    assert [lv.n_o for lv in H.levels[1:]] == [(1, 1, 3), (1, 1, 5)]
    assert its_max * 3 <= its_rel
