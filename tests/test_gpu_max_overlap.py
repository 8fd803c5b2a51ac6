"""GPU parity of the "max" overlap of the anisotropic study (Section 4.2,
Table 2): delta_O,i = min(max_j 0.08 dx_j, dx_i), a different N_O per
direction, strips up to a whole neighbour element (non-cubic subdomains with
lines of up to 3 (P+1) nodes), weights normalised over the covering
subdomains.  Same tolerances as the other parity tests: 1e-12 relative for
one application in FP64, 1e-10 through a V-cycle, 1e-4 for FP32."""
import math

import numpy as np
import pytest

from oracle.multigrid import Hierarchy, max_overlap_widths, solve_mgcg
from oracle.schwarz import SchwarzSmoother, max_width_layers, normalised_subdomain_1d
from oracle.sipg import Mesh, assemble, assemble_1d, weak_rhs
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


def study_lengths(ar):
    return (2 * math.pi * ar, 2 * math.pi * math.ceil(ar / 2), 2 * math.pi)


@pytest.fixture(scope="module")
def solvers(mg):
    cache = {}

    def get(ar, counts, P, precision="fp64", ns_growth=1):
        key = (ar, counts, P, precision, ns_growth)
        if key not in cache:
            cache[key] = mg.MGSolver(study_lengths(ar), counts, P, overlap_mode="max", overlap_frac=0.08,
                                     precision=precision, ns_growth=ns_growth)
        return cache[key]
    yield get
    for s in cache.values():
        s.close()


CASES = [(16, (4, 4, 4), 4), (48, (4, 4, 5), 4), (16, (4, 4, 4), 8), (3, (5, 4, 4), 8)]


@pytest.mark.parametrize("ar,counts,P", CASES)
def test_setup_tables_per_direction(solvers, ar, counts, P):
    """N_O, eigenpairs of the restricted 1D problems and the normalised weights
    of every level and direction."""
    s = solvers(ar, counts, P)
    mesh = Mesh(study_lengths(ar), counts)
    deltas = max_overlap_widths(mesh, 0.08)
    for l in range(1, s.L + 1):
        Pl = 2 ** l
        n = Pl + 1
        for d in range(3):
            no = max_width_layers(Pl, deltas[d])
            assert s.layers(l, d) == no
            Lo, Mo = assemble_1d(counts[d], mesh.lengths[d], Pl)
            Lo = Lo.toarray() if hasattr(Lo, "toarray") else Lo
            idx = np.arange(n - no, 2 * n + no)
            Ls, Ms = Lo[np.ix_(idx, idx)], Mo[idx]
            m = len(idx)
            S = s.get_table(l, d, 5).reshape(m, m)
            lam = s.get_table(l, d, 4)
            assert np.max(np.abs(S.T @ (Ms[:, None] * S) - np.eye(m))) < 1e-11
            assert np.max(np.abs(Ls @ S - Ms[:, None] * S * lam[None, :])) < 1e-11 * np.abs(Ls).max() * np.abs(S).max()
            _, _, w = normalised_subdomain_1d(Pl, no, deltas[d])
            np.testing.assert_allclose(s.get_table(l, d, 6), w, atol=1e-15)


@pytest.mark.parametrize("ar,counts,P", CASES)
def test_smooth_fp64(solvers, ar, counts, P):
    s = solvers(ar, counts, P)
    mesh = Mesh(study_lengths(ar), counts)
    A = assemble(mesh, P)
    deltas = max_overlap_widths(mesh, 0.08)
    n_os = tuple(max_width_layers(P, d) for d in deltas)
    sm = SchwarzSmoother(A, mesh, P, n_os, deltas)
    u = inputs.gaussian(A.shape[0], 4)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 5))
    ref = sm.correction(f - A @ u)
    ut = cuda(u)
    s.smooth(ut, cuda(f), nsteps=1)
    assert rel_err(host(ut) - u, ref) < FP64_TOL


def test_smooth_fp32(solvers):
    import torch
    ar, counts, P = 48, (4, 4, 5), 4
    s = solvers(ar, counts, P, precision="mixed")
    mesh = Mesh(study_lengths(ar), counts)
    A = assemble(mesh, P)
    deltas = max_overlap_widths(mesh, 0.08)
    sm = SchwarzSmoother(A, mesh, P, tuple(max_width_layers(P, d) for d in deltas), deltas)
    u = inputs.gaussian(A.shape[0], 8).astype(np.float32).astype(np.float64)
    f = weak_rhs(mesh, P, inputs.gaussian(A.shape[0], 9)).astype(np.float32).astype(np.float64)
    ref = sm.correction(f - A @ u)
    ut = cuda(u, torch.float32)
    s.smooth(ut, cuda(f, torch.float32))
    assert rel_err(host(ut) - u, ref) < 1e-4


@pytest.mark.parametrize("ar,counts,P", [(16, (4, 4, 4), 4), (16, (4, 4, 4), 8)])
def test_variable_vcycle(solvers, ar, counts, P):
    """One variable V-cycle N_s,l = (1,1) x 3^(L-l) with the max overlap."""
    s = solvers(ar, counts, P, ns_growth=3)
    mesh = Mesh(study_lengths(ar), counts)
    H = Hierarchy(mesh, P, max_frac=0.08)
    u = inputs.gaussian(H.A.shape[0], 16)
    f = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 17))
    ref = H.vcycle(u, f, 1, 1, 3)
    ut = cuda(u)
    s.vcycle(ut, cuda(f))
    assert rel_err(host(ut), ref) < 1e-10


def test_mgcg_solve_matches_oracle(solvers):
    """MG-CG with the variable cycle ("0.08 max; 1,1, var") at AR = 16."""
    ar, counts, P = 16, (4, 4, 4), 4
    s = solvers(ar, counts, P, ns_growth=3)
    mesh = Mesh(study_lengths(ar), counts)
    H = Hierarchy(mesh, P, max_frac=0.08)
    b = inputs.gaussian(H.A.shape[0], 2)
    b -= b.mean()
    uo, ito, ho = solve_mgcg(H, b, tol=1e-10, maxit=200, growth=3)
    ug, itg, rel, hg = s.solve(cuda(b), tol=1e-10, use_cg=True, maxit=200)
    assert abs(itg - ito) <= 1
    k = min(len(hg), len(ho))
    ho = np.asarray(ho)
    assert np.all(np.abs(hg[:k] - ho[:k]) <= 1e-6 * ho[:k] + 1e-14 * ho[0])
    assert rel_err(host(ug), uo) < 1e-8


def test_full_element_strip_needs_four_elements(mg):
    """A direction whose strip covers the whole neighbour element with only
    three elements would couple the two strips through the periodic boundary:
    rejected at setup."""
    with pytest.raises(Exception):
        mg.MGSolver(study_lengths(48), (4, 4, 3), 4, overlap_mode="max", overlap_frac=0.08)
