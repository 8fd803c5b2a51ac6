"""The per-level autotuner (mg_opts.autotune): mg_bind_workspace times the
kernel variants of every level's smoother, operator and scatter and keeps
the faster; whichever it keeps, the solve reaches the tolerance and agrees
with the untuned solve to rounding (the variants compute the same sums, in
the same order for the scatter, up to the FMA contraction of the others)."""
import numpy as np
import pytest

from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,outer", [("mixed", "all"), ("fp64", False), ("df64", False)])
def test_autotuned_solve_matches_default(mg, precision, outer):
    import torch
    lengths, counts, P = (2.0, 1.0, 1.0), (12, 8, 8), 8
    kw = dict(precision=precision, outer_df64=outer)
    s0 = mg.MGSolver(lengths, counts, P, **kw)
    s1 = mg.MGSolver(lengths, counts, P, autotune=True, **kw)
    for l in range(1, s1.L + 1):
        v = s1.kernel_variants(l)
        assert set(v.values()) <= {0, 1}, v
        assert s0.kernel_variants(l) == {"fdm": 0, "sipg": 0, "scatter": 0}
    b = s0.rhs(torch.tensor(inputs.gaussian(s0.num_dofs(), 41), device=s0.device))
    use_cg = precision == "mixed"
    u0, it0, rel0, _ = s0.solve(b, tol=1e-10, use_cg=use_cg)
    u1, it1, rel1, _ = s1.solve(b, tol=1e-10, use_cg=use_cg)
    assert rel0 <= 1e-10 and rel1 <= 1e-10 and abs(it0 - it1) <= 1
    a, c = u0.cpu().numpy(), u1.cpu().numpy()
    assert np.max(np.abs(a - c)) <= 1e-8 * np.max(np.abs(a))
    s0.close()
    s1.close()
