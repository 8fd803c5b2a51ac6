"""Pins of the oracle on graded meshes (element widths varying along each axis).

Graded meshes extend the paper (its grids are uniform, Section 4): the same
SIPG form (Section 2, Eq. ip) applied element by element, the subdomain solves
of Section 3.1 on subdomains whose restricted matrices now differ from one
element to the next.  The pins tie the graded oracle to closed forms and
invariants: equal widths reproduce the uniform matrices, the 3D assembly is the
Kronecker sum of the 1D factors (Eq. A), the 1D eigenvalues and the 3D L2 error
converge at the orders of the uniform mesh, the face penalty keeps the form
coercive down to the uniform threshold, and fast diagonalisation with one
eigenbasis per element line equals the direct subdomain solve.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spl

from oracle.gll import gll_nodes, lagrange_eval
from oracle.multigrid import Hierarchy, convergence_rate, solve_mg, solve_mgcg
from oracle.schwarz import subdomain_indices, subdomain_1d, layer_delta
from oracle.sipg import (Mesh, assemble, assemble_1d, assemble_1d_graded, local_index, mass_diagonal,
                         node_coordinates, weak_rhs)
from paper_1612_04796_gb300 import inputs


def graded_widths(count, length, ratio, seed):
    """Seeded widths of `count` elements summing to `length`, neighbouring
    widths differing by up to a factor `ratio`."""
    rng = np.random.default_rng(seed)
    w = np.exp(rng.uniform(-0.5 * math.log(ratio), 0.5 * math.log(ratio), size=count))
    return w * (length / w.sum())


def split(widths):
    """Every element cut into two halves (the grading pattern is kept)."""
    return np.repeat(np.asarray(widths) / 2.0, 2)


def kron_operator_graded(mesh, P, factor=2.0):
    """Eq. (A) from the graded 1D factors, permuted to element-blocked numbering."""
    n = P + 1
    Ls, Ms = [], []
    for d in range(3):
        L, M = assemble_1d_graded(mesh.widths[d], P, factor)
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


def small_graded_mesh(seed=7, counts=(3, 4, 3), ratio=3.0):
    lengths = (1.0, 2.0, 0.5)
    return Mesh(widths=[graded_widths(counts[d], lengths[d], ratio, seed + d) for d in range(3)])


@pytest.mark.parametrize("P", [1, 2, 4])
def test_equal_widths_reproduce_the_uniform_mesh(P):
    uni = Mesh((1.0, 2.0, 0.5), (3, 4, 2))
    gra = Mesh(widths=[np.full(3, 1.0 / 3), np.full(4, 0.5), np.full(2, 0.25)])
    A, Ag = assemble(uni, P), assemble(gra, P)
    assert abs(A - Ag).max() <= 1e-13 * abs(A).max()
    assert np.allclose(mass_diagonal(uni, P), mass_diagonal(gra, P), rtol=1e-15, atol=0)
    for a, b in zip(node_coordinates(uni, P), node_coordinates(gra, P)):
        assert np.allclose(a, b, rtol=0, atol=1e-15)
    L, M = assemble_1d(4, 2.0, P)
    Lg, Mg = assemble_1d_graded(np.full(4, 0.5), P)
    assert np.max(np.abs(L - Lg)) <= 1e-13 * np.max(np.abs(L)) and np.allclose(M, Mg, rtol=1e-15)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_graded_matrix_is_symmetric_psd_with_constant_nullspace(P):
    mesh = small_graded_mesh()
    A = assemble(mesh, P)
    scale = abs(A).max()
    assert abs(A - A.T).max() <= 1e-14 * scale
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) <= 1e-13 * scale
    if P <= 2:
        ev = np.linalg.eigvalsh(A.toarray())
        assert abs(ev[0]) < 1e-12 * ev[-1]
        assert ev[1] > 1e-6 * ev[-1]


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_graded_kronecker_form_eq_A(P):
    """The 3D element/face assembly on a graded tensor mesh equals
    Mz(x)My(x)Lx + Mz(x)Ly(x)Mx + Lz(x)My(x)Mx with the graded 1D factors."""
    mesh = small_graded_mesh(seed=11, counts=(3, 2, 4))
    A = assemble(mesh, P).toarray()
    Ak = kron_operator_graded(mesh, P)
    assert np.max(np.abs(A - Ak)) <= 1e-13 * np.max(np.abs(A))


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16])
def test_face_penalty_of_the_smaller_width_keeps_the_uniform_threshold(P):
    """With each face taking the penalty of its smaller neighbour, a graded line
    (neighbour ratios up to 16) stays positive semi-definite at the uniform
    threshold (factor 1); just below it, the graded line with equal widths is
    indefinite, as on the uniform mesh."""
    rng = np.random.default_rng(P)
    for _ in range(20):
        w = np.exp(rng.uniform(math.log(0.25), math.log(4.0), size=6))
        L, _ = assemble_1d_graded(w, P, factor=1.0)
        ev = np.linalg.eigvalsh(L)
        assert ev[0] > -1e-12 * ev[-1]
        assert np.max(np.abs(L @ np.ones(len(L)))) <= 1e-12 * ev[-1]
    L, _ = assemble_1d_graded(np.full(6, 0.5), P, factor=0.999)
    ev = np.linalg.eigvalsh(L)
    assert ev[0] < -1e-10 * ev[-1]


@pytest.mark.parametrize("P", [1, 2, 3])
def test_graded_1d_eigenvalues_converge_at_order_2p(P):
    """On a periodic graded interval of length l the lowest nonzero
    generalised eigenvalues approach (2 pi / l)^2 with error O(h^(2P)) when
    every element is halved."""
    l = 3.0
    exact = (2 * math.pi / l) ** 2
    w = graded_widths(8, l, 3.0, seed=5)
    errs = []
    for widths in (w, split(w)):
        L, M = assemble_1d_graded(widths, P)
        ev = sla.eigh(L, np.diag(M), eigvals_only=True)
        assert abs(ev[0]) < 1e-10 and ev[1] > 0
        errs.append(abs(0.5 * (ev[1] + ev[2]) - exact) / exact)
    order = math.log2(errs[0] / errs[1])
    assert 2 * P - 0.5 < order < 2 * P + 0.8, (errs, order)


def _graded_l2_error(P, widths):
    mesh = Mesh(widths=widths)
    A = assemble(mesh, P)
    X, Y, Z = node_coordinates(mesh, P)
    _, f = inputs.sines(X, Y, Z)
    b = weak_rhs(mesh, P, f)
    u, info = spl.cg(A, b, rtol=1e-13, atol=0.0, maxiter=20000)
    assert info == 0
    xg, wg = np.polynomial.legendre.leggauss(P + 3)
    phi = lagrange_eval(gll_nodes(P), xg)
    U = u.reshape(-1, P + 1, P + 1, P + 1)
    Ug = np.einsum("ai,bj,ck,ekji->ecba", phi, phi, phi, U)
    ex, ey, ez = mesh.element_coords()
    q, hs = [], []
    for d, ed in enumerate((ex, ey, ez)):
        x0, h = mesh.origins(d)[ed], mesh.widths[d][ed]
        q.append(x0[:, None] + (xg[None, :] + 1) * h[:, None] / 2)
        hs.append(h)
    xq, yq, zq = q
    ue = (np.sin(2 * np.pi * zq)[:, :, None, None] * np.sin(2 * np.pi * yq)[:, None, :, None]
          * np.sin(2 * np.pi * xq)[:, None, None, :])
    W = ((wg[:, None, None] * wg[None, :, None] * wg[None, None, :])[None]
         * (hs[0] * hs[1] * hs[2] / 8)[:, None, None, None])
    err = Ug - ue
    err = err - np.sum(W * err) / np.sum(W)
    return math.sqrt(np.sum(W * err ** 2))


@pytest.mark.parametrize("P", [2, 3])
def test_graded_l2_convergence_order_p_plus_1(P):
    """Manufactured periodic solution sin 2 pi x sin 2 pi y sin 2 pi z on the
    unit cube with graded widths: halving every element divides the L2 error
    by about 2^(P+1)."""
    n = 4 if P == 2 else 3
    w = [graded_widths(n, 1.0, 2.5, seed=20 + d) for d in range(3)]
    e1 = _graded_l2_error(P, w)
    e2 = _graded_l2_error(P, [split(x) for x in w])
    order = math.log2(e1 / e2)
    assert P + 1 - 0.5 < order < P + 1 + 0.8, order


@pytest.mark.parametrize("P,n_o", [(2, 1), (4, 1), (4, 2), (8, 1)])
def test_graded_fdm_with_per_line_eigenbases_equals_direct_solve(P, n_o):
    """For every subdomain of a graded mesh, A_ss (from the 3D assembly) is
    inverted exactly by fast diagonalisation with the eigenbases of the
    restricted graded 1D lines through its element (L_s S = M_s S Lambda)."""
    mesh = small_graded_mesh(seed=3, counts=(3, 3, 4), ratio=4.0)
    A = assemble(mesh, P)
    delta = layer_delta(P, n_o)
    idx, _ = subdomain_indices(mesh, P, n_o, delta)
    n = P + 1
    de, ii, _ = subdomain_1d(P, n_o, delta)
    ex, ey, ez = mesh.element_coords()
    one_d = [assemble_1d_graded(mesh.widths[d], P) for d in range(3)]
    rng = np.random.default_rng(P + n_o)
    for s in range(mesh.num_elements):
        Is = idx[s]
        Ass = A[Is][:, Is].toarray()
        fac = []
        for d, ed in enumerate((ex[s], ey[s], ez[s])):
            L, M = one_d[d]
            g = ((ed + de) % mesh.counts[d]) * n + ii
            lam, S = sla.eigh(L[np.ix_(g, g)], np.diag(M[g]))
            fac.append((S, lam))
        (Sx, lx), (Sy, ly), (Sz, lz) = fac
        r = rng.standard_normal(len(Is))
        m = len(de)
        R = r.reshape(m, m, m)  # (c, b, a)
        V = np.einsum("ap,bq,cr,cba->rqp", Sx, Sy, Sz, R)
        V /= lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
        U = np.einsum("ap,bq,cr,rqp->cba", Sx, Sy, Sz, V).ravel()
        direct = np.linalg.solve(Ass, r)
        assert np.max(np.abs(U - direct)) <= 1e-10 * np.max(np.abs(direct)), s


def test_graded_mg_and_mgcg_converge_like_the_uniform_mesh():
    """The V(1,1) cycle keeps its rate on a mildly graded mesh (neighbour
    ratios up to 2): MG and MG-CG reach 1e-10 in at most two cycles more than
    on the uniform mesh of the same counts."""
    P = 4
    counts = (4, 3, 4)
    uni = Mesh((1.0, 1.0, 1.0), counts)
    gra = Mesh(widths=[graded_widths(counts[d], 1.0, 2.0, seed=40 + d) for d in range(3)])
    its = {}
    for name, mesh in (("uniform", uni), ("graded", gra)):
        H = Hierarchy(mesh, P, n_o=1)
        f = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 9))
        _, it_mg, hist = solve_mg(H, f, tol=1e-10)
        _, it_cg, _ = solve_mgcg(H, f, tol=1e-10)
        assert hist[-1] <= 1e-10 * hist[0]
        its[name] = (it_mg, it_cg)
    assert its["graded"][0] <= its["uniform"][0] + 2, its
    assert its["graded"][1] <= its["uniform"][1] + 2, its


@pytest.mark.parametrize("graded,P,n_o", [(True, 4, 1), (True, 4, 2), (False, 4, 2), (True, 8, 1)])
def test_kron_fdm_correction_equals_direct_schwarz_correction(graded, P, n_o):
    """The fast-diagonalisation form of the smoother's correction (used where
    direct subdomain solves take too long) equals the direct solves of
    SchwarzSmoother on graded and uniform meshes."""
    from oracle.schwarz import SchwarzSmoother, kron_fdm_correction
    mesh = small_graded_mesh(seed=13, counts=(3, 4, 3), ratio=3.0) if graded else Mesh((1.0, 2.0, 0.5), (3, 4, 3))
    A = assemble(mesh, P)
    delta = layer_delta(P, n_o)
    r = np.random.default_rng(P + n_o).standard_normal(A.shape[0])
    ref = SchwarzSmoother(A, mesh, P, n_o, delta).correction(r)
    got = kron_fdm_correction(mesh, P, n_o, delta, r)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
