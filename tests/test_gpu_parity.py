"""GPU parity: every step of the hot path through the C ABI against the FP64
oracle on the same seeded inputs.

FP64 tolerance: 1e-12 relative (max-norm of the difference over the max-norm
of the reference) for single applications, as stated for the FP64 path; the
V-cycle and solves compare to 1e-10 because rounding differences grow through
a cycle.  FP32 kernels: 1e-5 relative (a few hundred FP32 ulps through
contractions of length <= 67)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.gll import gll_nodes, gll_weights, lagrange_eval
from oracle.multigrid import Hierarchy, convergence_rate, solve_mg, solve_mgcg
from oracle.schwarz import SchwarzSmoother, layer_delta, subdomain_1d
from oracle.sipg import Mesh, assemble, assemble_1d, node_coordinates, weak_rhs
from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


def cuda(x, dtype=None):
    import torch
    return torch.tensor(np.asarray(x), dtype=dtype or torch.float64, device="cuda")


def host(t):
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def solver_cache(mg):
    cache = {}

    def get(lengths, counts, P, overlap=1, **kw):
        key = (tuple(lengths), tuple(counts), P, overlap, tuple(sorted(kw.items())))
        if key not in cache:
            cache[key] = mg.MGSolver(lengths, counts, P, overlap=overlap, **kw)
        return cache[key]
    return get


# ---------------------------------------------------------------- setup tables
@pytest.mark.parametrize("P", [2, 4, 8, 16, 32])
def test_setup_basis_tables(solver_cache, P):
    s = solver_cache((1.0, 1.5, 0.7), (3, 4, 3), P)
    L = s.L
    np.testing.assert_allclose(s.get_table(L, 0, 0), gll_nodes(P), atol=1e-15)
    np.testing.assert_allclose(s.get_table(L, 0, 1), gll_weights(P), rtol=1e-13)
    for d, (n_el, length) in enumerate(zip(s.counts, s.lengths)):
        Lo, Mo = assemble_1d(n_el, length, P)
        n = P + 1
        lee = s.get_table(L, d, 3).reshape(n, n)
        assert rel_err(lee, Lo[:n, :n]) < FP64_TOL
        np.testing.assert_allclose(s.get_table(L, d, 2), Mo[:n], rtol=1e-14)


@pytest.mark.parametrize("P,overlap", [(2, 1), (4, 2), (8, 1), (8, 5), (16, 4), (32, 1)])
def test_setup_subdomain_eigenproblem(solver_cache, P, overlap):
    """S^T M_s S = I and L_s S = M_s S Lambda with the oracle's restricted 1D
    matrices; eigenvalues equal scipy's generalised eigh; weights equal the
    oracle's."""
    s = solver_cache((1.0, 1.5, 0.7), (3, 4, 3), P, overlap=overlap)
    L = s.L
    no = s.layers(L)
    n = P + 1
    for d, (n_el, length) in enumerate(zip(s.counts, s.lengths)):
        Lo, Mo = assemble_1d(n_el, length, P)
        idx = np.arange(n - no, 2 * n + no)
        Ls, Ms = Lo[np.ix_(idx, idx)], Mo[idx]
        m = len(idx)
        lam = s.get_table(L, d, 4)
        S = s.get_table(L, d, 5).reshape(m, m)
        scale = np.abs(Ls).max()
        assert np.max(np.abs(S.T @ (Ms[:, None] * S) - np.eye(m))) < 1e-12
        assert np.max(np.abs(Ls @ S - Ms[:, None] * S * lam[None, :])) < 1e-12 * scale * np.abs(S).max()
        ref = sla.eigh(Ls, np.diag(Ms), eigvals_only=True)
        np.testing.assert_allclose(np.sort(lam), ref, rtol=1e-11)
        _, _, w = subdomain_1d(P, no, layer_delta(P, no))
        np.testing.assert_allclose(s.get_table(L, d, 6), w, atol=1e-15)


@pytest.mark.parametrize("P", [2, 4, 8, 16, 32])
def test_setup_interpolation(solver_cache, P):
    s = solver_cache((1.0, 1.0, 1.0), (3, 3, 3), P)
    J = s.get_table(s.L, 0, 7).reshape(P + 1, P // 2 + 1)
    ref = lagrange_eval(gll_nodes(P // 2), gll_nodes(P))
    assert rel_err(J, ref) < 1e-13


@pytest.mark.parametrize("counts", [(3, 4, 5), (8, 3, 6)])
def test_setup_coarse_eigenbasis(solver_cache, counts):
    s = solver_cache((2.0, 1.0, 0.5), counts, 2)
    for d in range(3):
        Lo, Mo = assemble_1d(counts[d], s.lengths[d], 1)
        Ng = 2 * counts[d]
        lam = s.get_table(0, d, 8)
        Q = s.get_table(0, d, 9).reshape(Ng, Ng)
        assert np.max(np.abs(Q.T @ (Mo[:, None] * Q) - np.eye(Ng))) < 1e-12
        ref = sla.eigh(Lo, np.diag(Mo), eigvals_only=True)
        np.testing.assert_allclose(np.sort(lam), ref, atol=1e-11 * ref.max())


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("P,counts", [(2, (3, 4, 5)), (4, (3, 4, 5)), (8, (4, 3, 3)), (16, (3, 3, 3))])
def test_apply_sipg_fp64(solver_cache, P, counts):
    lengths = (1.0, 1.5, 0.7)
    s = solver_cache(lengths, counts, P)
    A = assemble(Mesh(lengths, counts), P)
    u = inputs.gaussian(A.shape[0], 1)
    got = host(s.apply_sipg(cuda(u)))
    assert rel_err(got, A @ u) < FP64_TOL
    f = inputs.gaussian(A.shape[0], 2)
    got_r = host(s.residual(cuda(u), cuda(f)))
    assert rel_err(got_r, f - A @ u) < FP64_TOL


def test_apply_sipg_all_levels(solver_cache):
    lengths, counts = (1.0, 1.5, 0.7), (3, 4, 3)
    s = solver_cache(lengths, counts, 8)
    mesh = Mesh(lengths, counts)
    for l in range(s.L + 1):
        A = assemble(mesh, 2 ** l)
        u = inputs.gaussian(A.shape[0], 10 + l)
        assert rel_err(host(s.apply_sipg(cuda(u), level=l)), A @ u) < FP64_TOL


@pytest.mark.parametrize("P", [4, 8, 16])  # P = 16 on 60 elements: the direction-split kernels
def test_apply_sipg_fp32(solver_cache, P):
    import torch
    lengths, counts = (1.0, 1.5, 0.7), (3, 4, 5)
    s = solver_cache(lengths, counts, P)
    A = assemble(Mesh(lengths, counts), P)
    u = inputs.gaussian(A.shape[0], 3).astype(np.float32)
    got = host(s.apply_sipg(cuda(u, torch.float32)))
    assert rel_err(got, A @ u.astype(np.float64)) < 1e-5


# ---------------------------------------------------------------- smoother
@pytest.mark.parametrize("P,overlap", [(2, 1), (4, 0), (4, 1), (4, 2), (4, 3), (8, 1), (8, 3)])
def test_smooth_fp64(solver_cache, P, overlap):
    lengths, counts = (1.0, 1.5, 0.7), (3, 4, 3)
    s = solver_cache(lengths, counts, P, overlap=overlap)
    mesh = Mesh(lengths, counts)
    A = assemble(mesh, P)
    no = s.layers(s.L)
    sm = SchwarzSmoother(A, mesh, P, no, layer_delta(P, no))
    u = inputs.gaussian(A.shape[0], 4)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 5))
    ref = sm.correction(f - A @ u)
    ut = cuda(u)
    s.smooth(ut, cuda(f), nsteps=1)
    assert rel_err(host(ut) - u, ref) < FP64_TOL
    # second step from the updated iterate
    u1 = u + ref
    ref2 = sm.correction(f - A @ u1)
    u1t = cuda(u1)
    s.smooth(u1t, cuda(f), nsteps=1)
    assert rel_err(host(u1t) - u1, ref2) < FP64_TOL


@pytest.mark.parametrize("profile", ["quintic", "linear", "quintic_halves", "quintic_normalised"])
def test_smooth_width_overlap(solver_cache, profile):
    """delta_O = 0.08 dx at P = 8: N_O = 2, weights from the transition profile."""
    lengths, counts, P = (1.0, 1.0, 1.0), (3, 3, 4), 8
    s = solver_cache(lengths, counts, P, overlap_mode="width", overlap_frac=0.08, weight_profile=profile)
    assert s.layers(s.L) == 2
    mesh = Mesh(lengths, counts)
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, 2, 0.16, profile)
    u = inputs.gaussian(A.shape[0], 6)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 7))
    ref = sm.correction(f - A @ u)
    ut = cuda(u)
    s.smooth(ut, cuda(f))
    assert rel_err(host(ut) - u, ref) < FP64_TOL


def test_smooth_fp32(solver_cache):
    import torch
    lengths, counts, P = (1.0, 1.5, 0.7), (3, 4, 3), 4
    s = solver_cache(lengths, counts, P, overlap=1)
    mesh = Mesh(lengths, counts)
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, 1, layer_delta(P, 1))
    u = inputs.gaussian(A.shape[0], 8).astype(np.float32).astype(np.float64)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 9)).astype(np.float32).astype(np.float64)
    ref = sm.correction(f - A @ u)
    ut = cuda(u, torch.float32)
    s.smooth(ut, cuda(f, torch.float32))
    assert rel_err(host(ut) - u, ref) < 1e-4


# ---------------------------------------------------------------- transfers, coarse
@pytest.mark.parametrize("P", [2, 4, 8])
def test_restrict_and_prolong(solver_cache, P):
    lengths, counts = (1.0, 1.5, 0.7), (3, 4, 3)
    s = solver_cache(lengths, counts, P)
    H = Hierarchy(Mesh(lengths, counts), P)
    L = s.L
    A = H.levels[L].A
    u = inputs.gaussian(A.shape[0], 12)
    f = inputs.gaussian(A.shape[0], 13)
    got = host(s.restrict_residual(cuda(u), cuda(f)))
    assert rel_err(got, H.restrict(L, f - A @ u)) < FP64_TOL
    uc = inputs.gaussian(H.levels[L - 1].N, 14)
    ut = cuda(u)
    s.prolongate(cuda(uc), ut)
    assert rel_err(host(ut) - u, H.prolong(L, uc)) < FP64_TOL


@pytest.mark.parametrize("counts", [(3, 3, 3), (4, 3, 5), (6, 4, 3)])
def test_coarse_solve(solver_cache, counts):
    lengths = (2.0, 1.0, 0.5)
    s = solver_cache(lengths, counts, 2)
    H = Hierarchy(Mesh(lengths, counts), 2)
    f0 = inputs.gaussian(H.levels[0].N, 15)
    got = host(s.coarse_solve(cuda(f0)))
    assert rel_err(got, H.coarse_solve(f0)) < 1e-11
    assert abs(got.mean()) < 1e-14 * np.abs(got).max()


# ---------------------------------------------------------------- cycle and solves
@pytest.mark.parametrize("P,overlap", [(4, 1), (8, 1), (8, 2)])
def test_vcycle_fp64(solver_cache, P, overlap):
    lengths, counts = (1.0, 1.5, 0.7), (3, 3, 4)
    s = solver_cache(lengths, counts, P, overlap=overlap)
    mesh = Mesh(lengths, counts)
    H = Hierarchy(mesh, P, n_o=overlap)
    u = inputs.gaussian(H.A.shape[0], 16)
    f = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 17))
    ref = H.vcycle(u, f)
    ut = cuda(u)
    s.vcycle(ut, cuda(f))
    assert rel_err(host(ut), ref) < 1e-10


def test_solve_c1_manufactured_matches_oracle(solver_cache):
    """Unit cube, 4^3 elements, P = 4, N_O = 1, manufactured sines."""
    lengths, counts, P = (1.0, 1.0, 1.0), (4, 4, 4), 4
    s = solver_cache(lengths, counts, P)
    mesh = Mesh(lengths, counts)
    H = Hierarchy(mesh, P)
    X, Y, Z = node_coordinates(mesh, P)
    u_ex, f = inputs.sines(X, Y, Z)
    b = weak_rhs(mesh, P, f)
    uo, ito, ho = solve_mg(H, b, tol=1e-10)
    # GPU side: coordinates and weak rhs from the library itself
    xg, yg, zg = (host(t) for t in s.node_coords())
    _, fg = inputs.sines(xg, yg, zg)
    bg = s.rhs(cuda(fg))
    assert rel_err(host(bg), b) < FP64_TOL
    ug, itg, rel, hg = s.solve(bg, tol=1e-10)
    assert itg == ito
    # residual norms agree to 6 digits or down to the rounding floor of the
    # FP64 residual f - A u (~1e-16 of the initial residual)
    ho = np.asarray(ho)
    assert np.all(np.abs(hg - ho) <= 1e-6 * ho + 1e-15 * ho[0])
    assert rel_err(host(ug), uo) < 1e-9
    assert np.max(np.abs(host(ug) - (u_ex - u_ex.mean()))) < 5e-3


def test_solve_cg_matches_oracle(solver_cache):
    lengths, counts, P = (1.0, 1.0, 1.0), (4, 4, 4), 4
    s = solver_cache(lengths, counts, P)
    mesh = Mesh(lengths, counts)
    H = Hierarchy(mesh, P)
    b = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 18))
    uo, ito, ho = solve_mgcg(H, b, tol=1e-10)
    ug, itg, rel, hg = s.solve(cuda(b), tol=1e-10, use_cg=True)
    assert itg == ito
    ho = np.asarray(ho)
    assert np.all(np.abs(hg - ho) <= 1e-6 * ho + 1e-15 * ho[0])
    assert rel_err(host(ug), uo) < 1e-9


@pytest.mark.parametrize("use_cg", [False, True])
def test_mixed_precision_reaches_fp64_tolerance(mg, use_cg):
    """FP32 multigrid inside the FP64 outer iteration reaches 1e-10 on the true
    FP64 residual; the solution matches the FP64 oracle solution to the
    accuracy the tolerance implies."""
    lengths, counts, P = (1.0, 1.0, 1.0), (4, 4, 4), 8
    s = mg.MGSolver(lengths, counts, P, precision="mixed")
    mesh = Mesh(lengths, counts)
    H = Hierarchy(mesh, P)
    b = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 19))
    uo, ito, _ = (solve_mgcg if use_cg else solve_mg)(H, b, tol=1e-10)
    ug, itg, rel, hg = s.solve(cuda(b), tol=1e-10, use_cg=use_cg)
    u = host(ug)
    assert np.linalg.norm(b - H.A @ u) <= 1.01e-10 * np.linalg.norm(b)
    assert abs(itg - ito) <= 2
    assert rel_err(u, uo) < 1e-7
