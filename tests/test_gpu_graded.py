"""GPU parity on graded meshes (element widths varying along each axis).

Every step of the hot path through the C ABI (mg_setup_graded and the usual
entry points) against the FP64 oracle on the same graded meshes and seeded
inputs: the per-line setup tables (Section 2 in one dimension, Section 3.1
subdomain eigenproblems), the operator (Eq. A), the smoother, the coarse
solve, the V-cycle (Algorithm 1) and MG / MG-CG solves (Section 3.2).

Tolerances as in the uniform parity tests: 1e-12 relative (max-norm) for one
FP64 application, 1e-10 through a V-cycle, 1e-5 for FP32 kernels."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.multigrid import Hierarchy, solve_mg, solve_mgcg
from oracle.schwarz import SchwarzSmoother, layer_delta, subdomain_1d
from oracle.sipg import Mesh, assemble, assemble_1d_graded, node_coordinates, weak_rhs
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


def graded_widths(count, length, ratio, seed):
    """Seeded widths of `count` elements summing to `length`, neighbouring
    widths differing by up to a factor `ratio` (the recipe of the oracle pins)."""
    rng = np.random.default_rng(seed)
    w = np.exp(rng.uniform(-0.5 * math.log(ratio), 0.5 * math.log(ratio), size=count))
    return w * (length / w.sum())


def mesh_widths(counts, lengths=(1.0, 1.5, 0.7), ratio=3.0, seed=7):
    return [graded_widths(counts[d], lengths[d], ratio, seed + d) for d in range(3)]


@pytest.fixture(scope="module")
def gsolver(mg):
    cache = {}

    def get(widths, P, overlap=1, **kw):
        key = (tuple(tuple(np.round(w, 15)) for w in widths), P, overlap, tuple(sorted(kw.items())))
        if key not in cache:
            cache[key] = mg.MGSolver(None, None, P, overlap=overlap, widths=widths, **kw)
        return cache[key]
    return get


# ---------------------------------------------------------------- setup tables
@pytest.mark.parametrize("P,overlap", [(2, 1), (4, 2), (8, 1), (8, 3), (16, 4), (32, 1)])
def test_line_tables_match_the_graded_1d_problem(gsolver, P, overlap):
    """Per element line: the mass weights and the rows of L equal the oracle's
    graded 1D matrices; the subdomain eigenpairs satisfy S^T M_s S = I and
    L_s S = M_s S Lambda with the oracle's restricted lines, and the
    eigenvalues equal scipy's."""
    widths = mesh_widths((3, 4, 3))
    s = gsolver(widths, P, overlap)
    assert s.lib.mg_is_graded(s.ctx) == 1
    L = s.L
    n = P + 1
    no = s.layers(L)
    de, ii, _ = subdomain_1d(P, no, layer_delta(P, no))
    for d in range(3):
        Lo, Mo = assemble_1d_graded(widths[d], P)
        nd = len(widths[d])
        for e in range(nd):
            np.testing.assert_allclose(s.get_line_table(L, d, e, 0), Mo[e * n:(e + 1) * n], rtol=1e-14)
            blk = s.get_line_table(L, d, e, 1).reshape(3, n, n)
            rows = slice(e * n, (e + 1) * n)
            for b, off in enumerate((-1, 0, 1)):
                c = (e + off) % nd
                ref = Lo[rows, c * n:(c + 1) * n]
                assert np.max(np.abs(blk[b] - ref)) <= FP64_TOL * np.abs(Lo).max(), (d, e, off)
            g = ((e + de) % nd) * n + ii
            Ls, Ms = Lo[np.ix_(g, g)], Mo[g]
            m = len(g)
            lam = s.get_line_table(L, d, e, 2)
            S = s.get_line_table(L, d, e, 3).reshape(m, m)
            scale = np.abs(Ls).max()
            assert np.max(np.abs(S.T @ (Ms[:, None] * S) - np.eye(m))) < 1e-12
            assert np.max(np.abs(Ls @ S - Ms[:, None] * S * lam[None, :])) < 1e-12 * scale * np.abs(S).max()
            ref = sla.eigh(Ls, np.diag(Ms), eigvals_only=True)
            np.testing.assert_allclose(np.sort(lam), ref, rtol=1e-11, atol=1e-13 * ref.max())


def test_graded_coarse_eigenbasis(gsolver):
    widths = mesh_widths((5, 3, 4))
    s = gsolver(widths, 2)
    for d in range(3):
        Lo, Mo = assemble_1d_graded(widths[d], 1)
        Ng = 2 * len(widths[d])
        lam = s.get_table(0, d, 8)
        Q = s.get_table(0, d, 9).reshape(Ng, Ng)
        assert np.max(np.abs(Q.T @ (Mo[:, None] * Q) - np.eye(Ng))) < 1e-12
        ref = sla.eigh(Lo, np.diag(Mo), eigvals_only=True)
        np.testing.assert_allclose(np.sort(lam), ref, atol=1e-11 * ref.max())


# ---------------------------------------------------------------- coordinates, rhs
def test_graded_coordinates_and_rhs(gsolver):
    widths = mesh_widths((4, 3, 5))
    P = 4
    s = gsolver(widths, P)
    mesh = Mesh(widths=widths)
    X, Y, Z = node_coordinates(mesh, P)
    xg, yg, zg = (host(t) for t in s.node_coords())
    for a, b in ((xg, X), (yg, Y), (zg, Z)):
        assert np.max(np.abs(a - b)) < 1e-14
    _, f = inputs.sines(X, Y, Z, mesh.lengths)
    assert rel_err(host(s.rhs(cuda(f))), weak_rhs(mesh, P, f)) < FP64_TOL


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("P,counts", [(2, (3, 4, 5)), (4, (3, 4, 5)), (8, (4, 3, 3)), (16, (3, 3, 3))])
def test_graded_apply_sipg_fp64(gsolver, P, counts):
    widths = mesh_widths(counts)
    s = gsolver(widths, P)
    A = assemble(Mesh(widths=widths), P)
    u = inputs.gaussian(A.shape[0], 1)
    assert rel_err(host(s.apply_sipg(cuda(u))), A @ u) < FP64_TOL
    f = inputs.gaussian(A.shape[0], 2)
    assert rel_err(host(s.residual(cuda(u), cuda(f))), f - A @ u) < FP64_TOL


def test_graded_apply_sipg_p32_sampled(gsolver):
    """P = 32 on a graded 3^3 mesh: the rows of three elements (the oracle
    assembles only those)."""
    widths = mesh_widths((3, 3, 3))
    s = gsolver(widths, 32)
    rows = [0, 13, 26]
    A = assemble(Mesh(widths=widths), 32, row_elements=rows)
    u = inputs.gaussian(A.shape[0], 26)
    got = host(s.apply_sipg(cuda(u)))
    B = 33 ** 3
    idx = np.concatenate([np.arange(e * B, (e + 1) * B) for e in rows])
    assert rel_err(got[idx], (A @ u)[idx]) < FP64_TOL


def test_graded_apply_sipg_all_levels(gsolver):
    widths = mesh_widths((3, 4, 3))
    s = gsolver(widths, 8)
    mesh = Mesh(widths=widths)
    for l in range(s.L + 1):
        A = assemble(mesh, 2 ** l)
        u = inputs.gaussian(A.shape[0], 10 + l)
        assert rel_err(host(s.apply_sipg(cuda(u), level=l)), A @ u) < FP64_TOL


def test_graded_apply_sipg_grid_stride(gsolver):
    """8^3 elements at P = 8 (373,248 DOFs): more DOFs than the launch has
    threads, strongly graded (neighbour ratios up to 8)."""
    widths = [graded_widths(8, 1.0, 8.0, 50 + d) for d in range(3)]
    s = gsolver(widths, 8)
    mesh = Mesh(widths=widths)
    rows = [0, 7, 63, 100, 300, 511]
    A = assemble(mesh, 8, row_elements=rows)
    u = inputs.gaussian(A.shape[0], 20)
    got = host(s.apply_sipg(cuda(u)))
    ref = A @ u
    B = 9 ** 3
    idx = np.concatenate([np.arange(e * B, (e + 1) * B) for e in rows])
    assert rel_err(got[idx], ref[idx]) < FP64_TOL


@pytest.mark.parametrize("P", [4, 8])
def test_graded_apply_sipg_fp32(gsolver, P):
    import torch
    widths = mesh_widths((3, 4, 5))
    s = gsolver(widths, P)
    A = assemble(Mesh(widths=widths), P)
    u = inputs.gaussian(A.shape[0], 3).astype(np.float32)
    got = host(s.apply_sipg(cuda(u, torch.float32)))
    assert rel_err(got, A @ u.astype(np.float64)) < 1e-5


# ---------------------------------------------------------------- smoother
@pytest.mark.parametrize("P,overlap", [(2, 1), (4, 0), (4, 1), (4, 2), (4, 3), (8, 1), (8, 3)])
def test_graded_smooth_fp64(gsolver, P, overlap):
    widths = mesh_widths((3, 4, 3), ratio=4.0)
    s = gsolver(widths, P, overlap)
    mesh = Mesh(widths=widths)
    A = assemble(mesh, P)
    no = s.layers(s.L)
    sm = SchwarzSmoother(A, mesh, P, no, layer_delta(P, no))
    u = inputs.gaussian(A.shape[0], 4)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 5))
    ref = sm.correction(f - A @ u)
    ut = cuda(u)
    s.smooth(ut, cuda(f), nsteps=1)
    assert rel_err(host(ut) - u, ref) < FP64_TOL
    u1 = u + ref
    ref2 = sm.correction(f - A @ u1)
    u1t = cuda(u1)
    s.smooth(u1t, cuda(f), nsteps=1)
    assert rel_err(host(u1t) - u1, ref2) < FP64_TOL


@pytest.mark.parametrize("P,overlap,dtype", [(16, 5, "fp64"), (32, 1, "fp64"), (16, 5, "fp32")])
def test_graded_smooth_full_widths(gsolver, P, overlap, dtype):
    """The widest graded subdomains (m = 27 at P = 16, N_O = 5; m = 35 at
    P = 32), beyond the compile-time widths, on a graded 3^3 mesh: one
    smoothing step from u = 0 against the oracle's fast-diagonalisation form
    of the correction (pinned to the direct subdomain solves)."""
    import torch
    from oracle.schwarz import kron_fdm_correction
    widths = mesh_widths((3, 3, 3), ratio=3.0)
    s = gsolver(widths, P, overlap)
    mesh = Mesh(widths=widths)
    no = s.layers(s.L)
    assert 2 * no + P + 1 > 25
    N = s.num_dofs()
    f = inputs.gaussian(N, 33)
    ref = kron_fdm_correction(mesh, P, no, layer_delta(P, no), f)
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    ut = torch.zeros(N, dtype=tdt, device="cuda")
    s.smooth(ut, cuda(f, tdt))
    assert rel_err(host(ut), ref) < (FP64_TOL if dtype == "fp64" else 1e-4)


def test_graded_smooth_many_subdomains_per_block(gsolver):
    """11^3 elements at P = 2: more subdomains than the smoother launches
    blocks, so every block transforms several subdomains in turn."""
    widths = [graded_widths(11, 1.0, 3.0, 60 + d) for d in range(3)]
    P = 2
    s = gsolver(widths, P, 1)
    mesh = Mesh(widths=widths)
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, 1, layer_delta(P, 1))
    u = inputs.gaussian(A.shape[0], 21)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 22))
    ref = sm.correction(f - A @ u)
    ut = cuda(u)
    s.smooth(ut, cuda(f))
    assert rel_err(host(ut) - u, ref) < FP64_TOL


@pytest.mark.parametrize("P,overlap", [(4, 1), (8, 2)])
def test_graded_smooth_fp32(gsolver, P, overlap):
    import torch
    widths = mesh_widths((3, 4, 3))
    s = gsolver(widths, P, overlap)
    mesh = Mesh(widths=widths)
    A = assemble(mesh, P)
    no = s.layers(s.L)
    sm = SchwarzSmoother(A, mesh, P, no, layer_delta(P, no))
    u = inputs.gaussian(A.shape[0], 8).astype(np.float32).astype(np.float64)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 9)).astype(np.float32).astype(np.float64)
    ref = sm.correction(f - A @ u)
    ut = cuda(u, torch.float32)
    s.smooth(ut, cuda(f, torch.float32))
    assert rel_err(host(ut) - u, ref) < 1e-4


# ---------------------------------------------------------------- transfers, coarse
def test_graded_restrict_prolong_and_coarse_solve(gsolver):
    widths = mesh_widths((4, 3, 5))
    P = 4
    s = gsolver(widths, P)
    H = Hierarchy(Mesh(widths=widths), P)
    L = s.L
    A = H.levels[L].A
    u = inputs.gaussian(A.shape[0], 12)
    f = inputs.gaussian(A.shape[0], 13)
    assert rel_err(host(s.restrict_residual(cuda(u), cuda(f))), H.restrict(L, f - A @ u)) < FP64_TOL
    uc = inputs.gaussian(H.levels[L - 1].N, 14)
    ut = cuda(u)
    s.prolongate(cuda(uc), ut)
    assert rel_err(host(ut) - u, H.prolong(L, uc)) < FP64_TOL
    f0 = inputs.gaussian(H.levels[0].N, 15)
    got = host(s.coarse_solve(cuda(f0)))
    assert rel_err(got, H.coarse_solve(f0)) < 1e-11
    assert abs(got.mean()) < 1e-14 * np.abs(got).max()


# ---------------------------------------------------------------- cycle and solves
@pytest.mark.parametrize("P,overlap", [(4, 1), (8, 1), (8, 2)])
def test_graded_vcycle_fp64(gsolver, P, overlap):
    widths = mesh_widths((3, 3, 4))
    s = gsolver(widths, P, overlap)
    mesh = Mesh(widths=widths)
    H = Hierarchy(mesh, P, n_o=overlap)
    u = inputs.gaussian(H.A.shape[0], 16)
    f = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 17))
    ref = H.vcycle(u, f)
    ut = cuda(u)
    s.vcycle(ut, cuda(f))
    assert rel_err(host(ut), ref) < 1e-10


@pytest.mark.parametrize("use_cg", [False, True])
def test_graded_solve_matches_oracle(gsolver, use_cg):
    """MG and MG-CG on a graded 4^3 mesh at P = 4: same iteration count,
    residual histories to 6 digits, same solution."""
    widths = [graded_widths(4, 1.0, 2.5, 30 + d) for d in range(3)]
    P = 4
    s = gsolver(widths, P)
    mesh = Mesh(widths=widths)
    H = Hierarchy(mesh, P)
    b = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 18))
    uo, ito, ho = (solve_mgcg if use_cg else solve_mg)(H, b, tol=1e-10)
    ug, itg, rel, hg = s.solve(cuda(b), tol=1e-10, use_cg=use_cg)
    assert itg == ito
    ho = np.asarray(ho)
    assert np.all(np.abs(hg - ho) <= 1e-6 * ho + 1e-15 * ho[0])
    assert rel_err(host(ug), uo) < 1e-9


def test_graded_mixed_precision_reaches_fp64_tolerance(gsolver):
    widths = [graded_widths(4, 1.0, 2.5, 40 + d) for d in range(3)]
    P = 8
    s = gsolver(widths, P, precision="mixed")
    mesh = Mesh(widths=widths)
    H = Hierarchy(mesh, P)
    b = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 19))
    uo, ito, _ = solve_mgcg(H, b, tol=1e-10)
    ug, itg, rel, hg = s.solve(cuda(b), tol=1e-10, use_cg=True)
    u = host(ug)
    assert np.linalg.norm(b - H.A @ u) <= 1.01e-10 * np.linalg.norm(b)
    assert abs(itg - ito) <= 2
    assert rel_err(u, uo) < 1e-7


def test_graded_vcycle_fp32(gsolver):
    """The FP32 hierarchy's V-cycle on a graded mesh equals the FP64 oracle's
    cycle to FP32 accuracy."""
    import torch
    widths = mesh_widths((3, 3, 4))
    P = 8
    s = gsolver(widths, P, 1, precision="mixed")
    mesh = Mesh(widths=widths)
    H = Hierarchy(mesh, P, n_o=1)
    u = inputs.gaussian(H.A.shape[0], 30).astype(np.float32).astype(np.float64)
    f = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 31)).astype(np.float32).astype(np.float64)
    ref = H.vcycle(u, f)
    ut = cuda(u, torch.float32)
    s.vcycle(ut, cuda(f, torch.float32))
    assert rel_err(host(ut), ref) < 1e-4


def test_graded_apply_sipg_df64(gsolver):
    """The double-float operator (the outer operator of the mixed solve with
    a double-float outer iteration) on a graded mesh: about 48 significant
    bits against the FP64 oracle."""
    widths = mesh_widths((3, 4, 5))
    P = 8
    s = gsolver(widths, P, precision="mixed", outer_df64=True)
    A = assemble(Mesh(widths=widths), P)
    u = inputs.gaussian(A.shape[0], 32)
    assert rel_err(host(s.apply_sipg_df64(cuda(u))), A @ u) < 1e-12


@pytest.mark.parametrize("outer", [True, "all"])
def test_graded_mixed_with_double_float_outer_iteration(gsolver, outer):
    widths = [graded_widths(4, 1.0, 2.5, 40 + d) for d in range(3)]
    P = 8
    s = gsolver(widths, P, precision="mixed", outer_df64=outer)
    mesh = Mesh(widths=widths)
    A = assemble(mesh, P)
    b = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 19))
    ug, itg, rel, _ = s.solve(cuda(b), tol=1e-10, use_cg=True)
    u = host(ug)
    assert np.linalg.norm(b - A @ u) <= 1.01e-10 * np.linalg.norm(b)
    assert itg <= 14


def test_equal_widths_match_the_uniform_path(mg):
    """A graded context with equal widths runs the graded kernels; its V-cycle
    equals the uniform context's to rounding."""
    lengths, counts, P = (1.0, 1.5, 0.7), (3, 4, 3), 8
    su = mg.MGSolver(lengths, counts, P)
    sg = mg.MGSolver(None, None, P, widths=[np.full(counts[d], lengths[d] / counts[d]) for d in range(3)])
    n = su.num_dofs()
    u = inputs.gaussian(n, 23)
    f = inputs.gaussian(n, 24)
    f -= f.mean()
    a, b = cuda(u), cuda(u)
    su.vcycle(a, cuda(f))
    sg.vcycle(b, cuda(f))
    assert rel_err(host(b), host(a)) < 1e-11


def test_graded_full_size_solve(gsolver):
    """16^3 graded elements at P = 8 (2,985,984 DOFs, neighbour ratios up to 2):
    sampled operator rows equal the oracle's; MG and mixed MG-CG reach the
    1e-10 FP64 residual."""
    import torch
    widths = [graded_widths(16, 1.0, 2.0, 70 + d) for d in range(3)]
    P = 8
    s = gsolver(widths, P)
    mesh = Mesh(widths=widths)
    rows = [0, 15, 255, 2048, 4095]
    A = assemble(mesh, P, row_elements=rows)
    u = inputs.gaussian(A.shape[0], 25)
    got = host(s.apply_sipg(cuda(u)))
    B = 9 ** 3
    idx = np.concatenate([np.arange(e * B, (e + 1) * B) for e in rows])
    assert rel_err(got[idx], (A @ u)[idx]) < FP64_TOL
    xg, yg, zg = s.node_coords()
    f = torch.randn(s.num_dofs(), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    b = s.rhs(f)
    _, it, rel, _ = s.solve(b, tol=1e-10)
    assert rel <= 1e-10 and it <= 20
    sm = gsolver(widths, P, precision="mixed")
    um, itm, relm, _ = sm.solve(b, tol=1e-10, use_cg=True)
    r = s.residual(um, b)
    assert float(torch.linalg.norm(r)) <= 1.01e-10 * float(torch.linalg.norm(b))


def test_graded_rejects_unsupported_options(mg):
    widths = mesh_widths((3, 3, 3))
    for kw in ({"precision": "df64"}, {"precision": "mixed", "tensor_cores": True}, {"overlap_mode": "width"},
               {"autotune": True}):
        with pytest.raises(mg.MGError):
            mg.MGSolver(None, None, 4, widths=widths, **kw)
    with pytest.raises(mg.MGError):
        mg.MGSolver(None, None, 4, widths=[np.array([0.5, -0.1, 0.6]), widths[1], widths[2]])


def test_graded_largest_line_count(gsolver):
    """n_x = 256, the largest element count along a graded axis (the coarse
    eigenproblem of that axis, 512 x 512, is solved whole in one block):
    coarse solve and V-cycle at P = 2 equal the oracle's."""
    widths = [graded_widths(256, 8.0, 2.0, 80), graded_widths(3, 1.0, 2.0, 81), graded_widths(3, 0.5, 2.0, 82)]
    P = 2
    s = gsolver(widths, P)
    mesh = Mesh(widths=widths)
    H = Hierarchy(mesh, P)
    f0 = inputs.gaussian(H.levels[0].N, 27)
    got = host(s.coarse_solve(cuda(f0)))
    assert rel_err(got, H.coarse_solve(f0)) < 1e-10
    u = inputs.gaussian(H.A.shape[0], 28)
    f = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 29))
    ut = cuda(u)
    s.vcycle(ut, cuda(f))
    assert rel_err(host(ut), H.vcycle(u, f)) < 1e-10
