"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: sampled elements against the oracle on local patches, and properties
of the full solves (iteration counts against Table 1, true residual, zero
mean, bitwise determinism)."""
import numpy as np
import pytest

from paper_1612_04796_gb300 import inputs
from patches import oracle_operator_at, oracle_smooth_at

pytestmark = pytest.mark.gpu

CUBE16_P8 = dict(lengths=(1.0, 1.0, 1.0), counts=(16, 16, 16), P=8)      # 16^3 elements, P = 8: the bench workload
CUBE4_P32 = dict(lengths=(1.0, 1.0, 1.0), counts=(4, 4, 4), P=32)


def _cuda(x):
    import torch
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def cube16(mg):
    s = mg.MGSolver(CUBE16_P8["lengths"], CUBE16_P8["counts"], CUBE16_P8["P"])
    N = s.num_dofs()
    u = inputs.gaussian(N, 41)
    f = inputs.gaussian(N, 42)
    return s, u, f


def _elements(counts, k, seed):
    rng = np.random.default_rng(seed)
    Ne = counts[0] * counts[1] * counts[2]
    return [0, Ne - 1] + list(rng.choice(Ne, k, replace=False))


def test_cube16_p8_operator_sampled(cube16):
    s, u, _ = cube16
    Au = s.apply_sipg(_cuda(u)).cpu().numpy()
    n3 = 9 ** 3
    for e in _elements(CUBE16_P8["counts"], 3, 1):
        ref = oracle_operator_at(u, CUBE16_P8["lengths"], CUBE16_P8["counts"], 8, e)
        got = Au[e * n3:(e + 1) * n3]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12, e


def test_cube16_p8_smoother_sampled(cube16):
    s, u, f = cube16
    ut = _cuda(u)
    s.smooth(ut, _cuda(f))
    corr = ut.cpu().numpy() - u
    n3 = 9 ** 3
    for e in _elements(CUBE16_P8["counts"], 1, 2):
        ref = oracle_smooth_at(u, f, CUBE16_P8["lengths"], CUBE16_P8["counts"], 8, 1, e)
        got = corr[e * n3:(e + 1) * n3]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12, e


def test_cube16_p8_solve_properties(cube16, mg):
    """The bench solve: 12 V(1,1) cycles (Table 1 row 1, P = 8: rbar = 0.89,
    n10 = ceil(10 / 0.89) = 12), true FP64 residual <= 1e-10, zero mean, and
    bitwise identical on a rerun."""
    import torch
    s, _, _ = cube16
    N = s.num_dofs()
    b = s.rhs(_cuda(inputs.gaussian(N, 2)))
    u1, it1, rel1, hist = s.solve(b, tol=1e-10)
    assert it1 == 12
    true_rel = float(torch.linalg.norm(s.residual(u1, b)) / torch.linalg.norm(b))
    assert true_rel <= 1e-10
    assert abs(float(u1.sum())) <= 1e-12 * float(u1.abs().sum())
    rho = (hist[-1] / hist[0]) ** (1.0 / it1)
    assert abs(-np.log10(rho) - 0.89) < 0.15
    u2, it2, _, _ = s.solve(b, tol=1e-10)
    assert it2 == it1 and torch.equal(u1, u2)
    # the mixed path on the same problem reaches the same tolerance
    sm = mg.MGSolver(CUBE16_P8["lengths"], CUBE16_P8["counts"], CUBE16_P8["P"], precision="mixed")
    um, itm, _, _ = sm.solve(b, tol=1e-10, use_cg=True)
    assert float(torch.linalg.norm(s.residual(um, b)) / torch.linalg.norm(b)) <= 1.01e-10
    assert float((um - u1).abs().max() / u1.abs().max()) < 1e-8


def test_cube4_p32_operator_sampled(mg):
    s = mg.MGSolver(CUBE4_P32["lengths"], CUBE4_P32["counts"], CUBE4_P32["P"])
    u = inputs.gaussian(s.num_dofs(), 43)
    Au = s.apply_sipg(_cuda(u)).cpu().numpy()
    n3 = 33 ** 3
    for e in (0, 37):
        ref = oracle_operator_at(u, CUBE4_P32["lengths"], CUBE4_P32["counts"], 32, e)
        got = Au[e * n3:(e + 1) * n3]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12, e


def test_p16_fp64_operator_one_thread_per_line(mg):
    """The FP64 operator at P = 16 on a mesh with enough lines for one thread
    per line (8x6x6 elements, 83k lines per direction; the 48x8x8 box runs
    this form): sampled elements against the oracle, 1e-12."""
    lengths, counts, P = (1.0, 1.5, 0.7), (8, 6, 6), 16
    s = mg.MGSolver(lengths, counts, P)
    u = inputs.gaussian(s.num_dofs(), 47)
    Au = s.apply_sipg(_cuda(u)).cpu().numpy()
    s.close()
    n3 = 17 ** 3
    for e in (0, 100, 287):
        ref = oracle_operator_at(u, lengths, counts, 16, e)
        got = Au[e * n3:(e + 1) * n3]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12, e


@pytest.mark.parametrize("arith", ["fp32", "df64"])
def test_cube4_p32_operator_sampled_fp32_df64(mg, arith):
    """The operator of the mixed solve at P = 32 (n = 33 on 64 elements: the
    direction-split kernels with the 1D coefficients as kernel parameters) in
    FP32 (the multigrid's residuals; 1e-5 of the element's largest entry) and
    in double-float (the outer iteration's A p; 1e-12)."""
    import torch
    s = mg.MGSolver(CUBE4_P32["lengths"], CUBE4_P32["counts"], CUBE4_P32["P"], precision="mixed",
                    outer_df64=True)
    u = inputs.gaussian(s.num_dofs(), 44)
    if arith == "fp32":
        u = u.astype(np.float32).astype(np.float64)
        Au = s.apply_sipg(torch.tensor(u, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    else:
        Au = s.apply_sipg_df64(_cuda(u)).cpu().numpy()
    s.close()
    n3 = 33 ** 3
    for e in (0, 37, 63):
        ref = oracle_operator_at(u, CUBE4_P32["lengths"], CUBE4_P32["counts"], 32, e)
        got = Au[e * n3:(e + 1) * n3]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < (1e-5 if arith == "fp32" else 1e-12), (e, arith)


def test_cube4_p32_mixed_solve_reaches_tolerance(mg):
    """High order (P = 32): FP32 V-cycle inside FP64 CG reaches 1e-10 on the
    true FP64 residual; MG-CG takes about ceil(10 / 0.52) = 20 iterations
    (Table 1 row 2, P = 32)."""
    import torch
    s = mg.MGSolver(CUBE4_P32["lengths"], CUBE4_P32["counts"], CUBE4_P32["P"], precision="mixed")
    s64 = mg.MGSolver(CUBE4_P32["lengths"], CUBE4_P32["counts"], CUBE4_P32["P"])
    N = s.num_dofs()
    x, y, z = (t.cpu().numpy() for t in s.node_coords())
    f = inputs.eval_fourier(inputs.fourier_modes(4), x, y, z)
    b = s.rhs(_cuda(f))
    u, its, rel, _ = s.solve(b, tol=1e-10, use_cg=True, maxit=60)
    assert float(torch.linalg.norm(s64.residual(u, b)) / torch.linalg.norm(b)) <= 1.01e-10
    assert 14 <= its <= 26


def test_cube16_p8_double_float_solves(cube16, mg):
    """The bench problem with the multigrid in double-float: the FP64 path's
    12 cycles and a solution within 1e-12 of the FP64 one; and the mixed
    solve with the double-float outer operator: the true FP64 residual
    reaches 1e-10 in the same 9 iterations as with the FP64 outer operator."""
    import torch
    s, _, _ = cube16
    N = s.num_dofs()
    b = s.rhs(_cuda(inputs.gaussian(N, 2)))
    u64, it64, _, _ = s.solve(b, tol=1e-10)
    sd = mg.MGSolver(CUBE16_P8["lengths"], CUBE16_P8["counts"], CUBE16_P8["P"], precision="df64")
    ud, itd, _, _ = sd.solve(b, tol=1e-10)
    assert itd == it64
    assert float(torch.linalg.norm(s.residual(ud, b)) / torch.linalg.norm(b)) <= 1e-10
    assert float((ud - u64).abs().max() / u64.abs().max()) < 1e-12
    sd.close()
    its = []
    for df in (False, True):
        sm = mg.MGSolver(CUBE16_P8["lengths"], CUBE16_P8["counts"], CUBE16_P8["P"], precision="mixed",
                         outer_df64=df)
        um, itm, _, _ = sm.solve(b, tol=1e-10, use_cg=True)
        assert float(torch.linalg.norm(s.residual(um, b)) / torch.linalg.norm(b)) <= 1.01e-10
        its.append(itm)
        sm.close()
    assert its[0] == its[1]


@pytest.mark.parametrize("ctx_precision", ["fp64", "mixed"])
def test_p32_fp32_vcycle_matches_fp64(mg, ctx_precision):
    """One FP32 V-cycle at P = 32 (3^3 elements; the transfers between the
    P = 32 and P = 16 levels with the 1D matrix as kernel parameters, and in a
    mixed context the split smoother and the direction-split operator)
    against the FP64 V-cycle, whose kernels are separate code: equal to FP32
    rounding (1e-4 of the largest entry of the result)."""
    import torch
    lengths, counts, P = (1.0, 1.5, 0.7), (3, 3, 3), 32
    s64 = mg.MGSolver(lengths, counts, P)
    s32 = s64 if ctx_precision == "fp64" else mg.MGSolver(lengths, counts, P, precision="mixed")
    N = s64.num_dofs()
    u = inputs.gaussian(N, 45).astype(np.float32).astype(np.float64)
    f = inputs.gaussian(N, 46).astype(np.float32).astype(np.float64)
    u64 = s64.vcycle(_cuda(u), _cuda(f)).cpu().numpy()
    ut = torch.tensor(u, dtype=torch.float32, device="cuda")
    u32 = s32.vcycle(ut, torch.tensor(f, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    err = np.max(np.abs(u32 - u64)) / np.max(np.abs(u64))
    assert err < 1e-4, err
    if s32 is not s64:
        s32.close()
    s64.close()
