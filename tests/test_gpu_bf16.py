"""Precision study for BF16 and FP8 contractions in the FP32 smoother
(mg_opts.fdm_operands): every line entering a 1D product and the 1D factors
rounded to BF16 (8 significant bits) or to FP8 E4M3 (4 significant bits,
after a power-of-two scale per line and per factor column: "scaled
eigenbases"), FP32 accumulation -- what BF16 / FP8 tensor-core contractions
compute, run on the CUDA cores.

The subdomain solve (Section 3.1) then carries about 2^-8 (BF16) or 2^-4
(FP8) relative error per contraction; six contractions and the
small-eigenvalue modes that dominate the correction give a smoother error of
order 1e-2 (BF16; bound 5e-2) or 1e-1 (FP8; bound 0.3) against the oracle,
against 1e-5 for FP32 operands.  The double-float outer iteration still
reaches the 1e-10 true residual, with the same number of iterations or one
more for BF16 and a few more for FP8."""
import numpy as np
import pytest

from oracle.schwarz import SchwarzSmoother, layer_delta
from oracle.sipg import Mesh, assemble
from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu

BOUNDS = {"fp32": (0.0, 1e-5), "bf16": (1e-4, 5e-2), "fp8": (1e-2, 0.3)}


def test_operand_study_smoother_error(mg):
    import torch
    lengths, counts, P = (1.0, 1.5, 0.7), (3, 4, 3), 8
    mesh = Mesh(lengths, counts)
    A = assemble(mesh, P)
    N = A.shape[0]
    u = inputs.gaussian(N, 70).astype(np.float32).astype(np.float64)
    f = inputs.gaussian(N, 71).astype(np.float32).astype(np.float64)
    ref = SchwarzSmoother(A, mesh, P, 1, layer_delta(P, 1)).correction(f - A @ u)
    errs = {}
    for op in BOUNDS:
        s = mg.MGSolver(lengths, counts, P, precision="mixed", fdm_operands=op)
        ut = torch.tensor(u, dtype=torch.float32, device="cuda")
        s.smooth(ut, torch.tensor(f, dtype=torch.float32, device="cuda"))
        got = ut.double().cpu().numpy() - u
        errs[op] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        s.close()
    for op, (lo, hi) in BOUNDS.items():
        assert lo <= errs[op] < hi, errs
    # the legacy switch is the BF16 study
    s = mg.MGSolver(lengths, counts, P, precision="mixed", fdm_bf16=True)
    assert s.opts.fdm_operands == 1
    s.close()


def test_operand_study_mgcg_reaches_tolerance(mg):
    import torch
    lengths, counts, P = (1.0, 1.0, 1.0), (8, 8, 8), 8
    its = {}
    for op in BOUNDS:
        s = mg.MGSolver(lengths, counts, P, precision="mixed", outer_df64="all", fdm_operands=op)
        b = s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), 72), device="cuda"))
        u, it, rel, _ = s.solve(b, tol=1e-10, use_cg=True)
        s64 = mg.MGSolver(lengths, counts, P)
        true = float(torch.linalg.norm(s64.residual(u, b)) / torch.linalg.norm(b))
        assert true <= 1e-10 * (1 + 1e-6), (op, true)
        its[op] = it
        s.close()
        s64.close()
    assert its["fp32"] <= its["bf16"] <= its["fp32"] + 1, its
    assert its["bf16"] <= its["fp8"] <= its["fp32"] + 6, its
