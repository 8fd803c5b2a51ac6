"""GPU parity at the subdomain widths of the full-size configurations.

The smoother kernels are compiled for each odd width m = n + 2 N_O; these
tests compare every width the large configurations run with the FP64 oracle
(direct subdomain solves, Section 3.1), element by element:

* m = 17, 19, 21, 25: P = 16 with N_O = 0, 1, 2, 4 (the 48x8x8, P = 16
  configuration runs 19, 21 and 25) on a 3x4x3 periodic box with three
  different element widths, so that the x, y and z factors differ;
* m = 35: P = 32 with N_O = 1 (the 4^3, P = 32 configuration), against
  sampled values that tests/golden/make_smoother_wide.py stored from the
  oracle (a direct solve at m = 35 takes minutes and 15 GB).

FP64 and double-float arithmetic, FP32, and FP32 with the contractions on
the tensor cores (TF32 inputs, FP32 accumulation).  Tolerances (max-norm of
the difference over the max-norm of the oracle's correction): FP64 1e-12
(the FP64 path's bound for one application); double-float 1e-10 (about 48
significant bits per operation); FP32 1e-5 (contractions of length <= 35 in
each of six passes, a few hundred FP32 ulps); TF32 2e-2 in the max norm and
5e-3 in the 2-norm (10 fraction bits per contraction input through six
passes, as in the tensor-core tests at the smaller widths).

Also: the FP64 multigrid solve of the 6^3, P = 8 problem that bench.py times
for its CPU baseline (same cycles, same residual history as the oracle), and
MG-CG at P = 16 on a 3^3 mesh."""
import json
import os

import numpy as np
import pytest

from oracle.multigrid import Hierarchy, solve_mg, solve_mgcg
from oracle.schwarz import SchwarzSmoother, layer_delta
from oracle.sipg import Mesh, assemble, weak_rhs
from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
LENGTHS = (1.0, 1.5, 0.7)
COUNTS = (3, 4, 3)
P16_LAYERS = [0, 1, 2, 4]  # m = 17, 19, 21, 25
TOL = {"fp64": 1e-12, "df64": 1e-10, "fp32": 1e-5, "tf32": 2e-2}
TF32_L2 = 5e-3


def rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got) - ref)) / np.max(np.abs(ref)))


def cuda(x, dtype=None):
    import torch
    return torch.tensor(np.asarray(x), dtype=dtype or torch.float64, device="cuda")


@pytest.fixture(scope="module")
def p16_case():
    """Oracle corrections at P = 16 for each N_O (inputs rounded to FP32 so
    that the FP32 kernel sees the same values)."""
    mesh = Mesh(LENGTHS, COUNTS)
    A = assemble(mesh, 16)
    N = A.shape[0]
    u = inputs.gaussian(N, 50).astype(np.float32).astype(np.float64)
    f = inputs.gaussian(N, 51).astype(np.float32).astype(np.float64)
    r = f - A @ u
    corr = {}
    for no in P16_LAYERS:
        sm = SchwarzSmoother(A, mesh, 16, no, layer_delta(16, no), check=4, dense_limit=16000)
        corr[no] = sm.correction(r)
    return u, f, corr


def gpu_smooth(mg, arith, lengths, counts, P, no, u, f):
    import torch
    tc = arith == "tf32"
    s = mg.MGSolver(lengths, counts, P, overlap=no, **(dict(precision="mixed", tensor_cores=True) if tc else {}))
    assert s.layers(s.L) == no
    if tc:
        assert s.fdm_tensor_cores(s.L) == 1  # the fine level's tiles fit the tensor-core kernel
    if arith in ("fp32", "tf32"):
        ut = cuda(u, torch.float32)
        s.smooth(ut, cuda(f, torch.float32))
    elif arith == "df64":
        ut = cuda(u)
        s.smooth_df64(ut, cuda(f))
    else:
        ut = cuda(u)
        s.smooth(ut, cuda(f))
    out = ut.double().cpu().numpy() - u
    s.close()
    return out


@pytest.mark.parametrize("arith", ["fp64", "df64", "fp32", "tf32"])
@pytest.mark.parametrize("no", P16_LAYERS)
def test_smooth_p16_widths(mg, p16_case, no, arith):
    u, f, corr = p16_case
    got = gpu_smooth(mg, arith, LENGTHS, COUNTS, 16, no, u, f)
    err = rel_err(got, corr[no])
    assert err < TOL[arith], (16 + 1 + 2 * no, arith, err)
    if arith == "tf32":
        e2 = float(np.linalg.norm(got - corr[no]) / np.linalg.norm(corr[no]))
        assert e2 < TF32_L2, (16 + 1 + 2 * no, e2)


@pytest.fixture(scope="module")
def m35_golden():
    with open(os.path.join(HERE, "golden", "smoother_p32_m35.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("arith", ["fp64", "df64", "fp32", "tf32"])
def test_smooth_m35_matches_stored_oracle(mg, m35_golden, arith):
    g = m35_golden
    c = g["case"]
    assert g["subdomain_width"] == 35
    N = g["dofs"]
    u = inputs.gaussian(N, c["seed_u"]).astype(np.float32).astype(np.float64)
    f = inputs.gaussian(N, c["seed_f"]).astype(np.float32).astype(np.float64)
    got = gpu_smooth(mg, arith, c["lengths"], c["elements"], c["P"], c["overlap_layers"], u, f)
    idx = np.asarray(g["index"])
    err = float(np.max(np.abs(got[idx] - np.asarray(g["value"]))) / g["correction_max_abs"])
    assert err < TOL[arith], (arith, err)
    # the whole correction has the oracle's size (every sampled value agrees, and
    # nothing outside the sample is wildly off)
    size_tol = TF32_L2 if arith == "tf32" else 10 * TOL[arith]
    assert abs(np.max(np.abs(got)) / g["correction_max_abs"] - 1.0) < max(size_tol, TOL[arith])
    assert abs(np.linalg.norm(got) / g["correction_norm2"] - 1.0) < size_tol
    if arith == "tf32":
        ref = np.asarray(g["value"])
        e2 = float(np.linalg.norm(got[idx] - ref) / np.linalg.norm(ref))
        assert e2 < TF32_L2, e2


def test_mg_solve_6cube_p8_matches_oracle(mg):
    """The problem bench.py solves with the CPU oracle for its baseline:
    unit cube, 6^3 elements, P = 8, N_O = 1, Gaussian f (seed 2), standalone
    V(1,1) cycles to 1e-10.  Same cycle count, residual norms to 6 digits (or
    the FP64 rounding floor), solutions within 1e-9."""
    lengths, counts, P = (1.0, 1.0, 1.0), (6, 6, 6), 8
    mesh = Mesh(lengths, counts)
    H = Hierarchy(mesh, P)
    b = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 2))
    uo, ito, ho = solve_mg(H, b, tol=1e-10)
    s = mg.MGSolver(lengths, counts, P)
    ug, itg, rel, hg = s.solve(cuda(b), tol=1e-10)
    u = ug.cpu().numpy()
    s.close()
    assert itg == ito
    ho = np.asarray(ho)
    assert np.all(np.abs(hg - ho) <= 1e-6 * ho + 1e-15 * ho[0])
    assert rel_err(u, uo) < 1e-9


def test_mgcg_p16_matches_oracle(mg):
    """MG-CG at P = 16 (five levels, m = 19 on the fine level) on a 3^3 box
    with three element widths: same iterations and residual history."""
    lengths, counts, P = LENGTHS, (3, 3, 3), 16
    mesh = Mesh(lengths, counts)
    H = Hierarchy(mesh, P)
    b = weak_rhs(mesh, P, inputs.gaussian(H.A.shape[0], 52))
    uo, ito, ho = solve_mgcg(H, b, tol=1e-10)
    s = mg.MGSolver(lengths, counts, P)
    ug, itg, rel, hg = s.solve(cuda(b), tol=1e-10, use_cg=True)
    u = ug.cpu().numpy()
    s.close()
    assert itg == ito
    ho = np.asarray(ho)
    assert np.all(np.abs(hg - ho) <= 1e-6 * ho + 1e-15 * ho[0])
    assert rel_err(u, uo) < 1e-9
