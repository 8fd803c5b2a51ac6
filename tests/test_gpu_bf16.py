"""Precision study for BF16 contractions in the FP32 smoother (mg_opts.fdm_bf16):
every line entering a 1D product and the 1D factors rounded to BF16 (8
significant bits), FP32 accumulation -- what BF16 tensor-core contractions
compute, run on the CUDA cores.

The subdomain solve (Section 3.1) then carries about 2^-8 relative error
per contraction; six contractions and the small-eigenvalue modes that
dominate the correction give a smoother error of order 1e-2 against the
oracle (bound here 5e-2, against 1e-5 for FP32 operands).  The FP64 / double-
float outer iteration still reaches the 1e-10 true residual."""
import numpy as np
import pytest

from oracle.schwarz import SchwarzSmoother, layer_delta
from oracle.sipg import Mesh, assemble
from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bf16_operand_smoother_error(mg):
    import torch
    lengths, counts, P = (1.0, 1.5, 0.7), (3, 4, 3), 8
    mesh = Mesh(lengths, counts)
    A = assemble(mesh, P)
    N = A.shape[0]
    u = inputs.gaussian(N, 70).astype(np.float32).astype(np.float64)
    f = inputs.gaussian(N, 71).astype(np.float32).astype(np.float64)
    ref = SchwarzSmoother(A, mesh, P, 1, layer_delta(P, 1)).correction(f - A @ u)
    errs = {}
    for bf in (False, True):
        s = mg.MGSolver(lengths, counts, P, precision="mixed", fdm_bf16=bf)
        ut = torch.tensor(u, dtype=torch.float32, device="cuda")
        s.smooth(ut, torch.tensor(f, dtype=torch.float32, device="cuda"))
        got = ut.double().cpu().numpy() - u
        errs[bf] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        s.close()
    assert errs[False] < 1e-5
    assert 1e-4 < errs[True] < 5e-2, errs


def test_bf16_operand_mgcg_reaches_tolerance(mg):
    import torch
    lengths, counts, P = (1.0, 1.0, 1.0), (8, 8, 8), 8
    its = {}
    for bf in (False, True):
        s = mg.MGSolver(lengths, counts, P, precision="mixed", outer_df64="all", fdm_bf16=bf)
        b = s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), 72), device="cuda"))
        u, it, rel, _ = s.solve(b, tol=1e-10, use_cg=True)
        s64 = mg.MGSolver(lengths, counts, P)
        true = float(torch.linalg.norm(s64.residual(u, b)) / torch.linalg.norm(b))
        assert true <= 1e-10 * (1 + 1e-6), (bf, true)
        its[bf] = it
        s.close()
        s64.close()
    assert its[True] >= its[False]
