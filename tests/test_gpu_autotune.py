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
        # the FP32 smoother has a third variant (its passes split over three kernels)
        assert v["fdm"] in ((0, 1, 2) if precision == "mixed" else (0, 1)) and v["sipg"] in (0, 1) \
            and v["scatter"] in (0, 1), v
        # defaults: the split FP32 smoother from m = 11 up (the P = 8 level here), else 0
        fdm0 = 2 if precision == "mixed" and l == s0.L else 0
        assert s0.kernel_variants(l) == {"fdm": fdm0, "sipg": 0, "scatter": 0}
    b = s0.rhs(torch.tensor(inputs.gaussian(s0.num_dofs(), 41), device=s0.device))
    use_cg = precision == "mixed"
    u0, it0, rel0, _ = s0.solve(b, tol=1e-10, use_cg=use_cg)
    u1, it1, rel1, _ = s1.solve(b, tol=1e-10, use_cg=use_cg)
    assert rel0 <= 1e-10 and rel1 <= 1e-10 and abs(it0 - it1) <= 1
    a, c = u0.cpu().numpy(), u1.cpu().numpy()
    assert np.max(np.abs(a - c)) <= 1e-8 * np.max(np.abs(a))
    s0.close()
    s1.close()


def test_split_smoother_matches_fused(mg):
    """On the 4^3, P = 32 mesh (64 subdomains) the mixed solver's levels of
    width m >= 11 default to the FP32 smoother split over three grid-wide
    kernels; it makes the products of the one-kernel smoother, line by line in
    the same order, so one smoothing step agrees with it to the last bit (or
    within an ulp where the compiler contracts differently) at m = 35, 19 and
    11."""
    import torch
    lengths, counts, P = (1.0, 1.0, 1.0), (4, 4, 4), 32
    sm = mg.MGSolver(lengths, counts, P, precision="mixed")
    s1 = mg.MGSolver(lengths, counts, P)  # FP64 context: FP32 smoothing steps use the one-kernel smoother
    assert [sm.kernel_variants(l)["fdm"] for l in (sm.L, sm.L - 1, sm.L - 2)] == [2, 2, 2]
    assert sm.kernel_variants(sm.L - 3)["fdm"] == 0  # m = 7: the one-kernel form
    for lev in (sm.L, sm.L - 1, sm.L - 2):
        N = sm.num_dofs(lev)
        u = torch.tensor(inputs.gaussian(N, 60 + lev), dtype=torch.float32, device=sm.device)
        f = torch.tensor(inputs.gaussian(N, 70 + lev), dtype=torch.float32, device=sm.device)
        ua, ub = u.clone(), u.clone()
        sm.smooth(ua, f, level=lev)
        s1.smooth(ub, f, level=lev)
        d = (ua - ub).abs().max().item() / (ub - u).abs().max().item()
        assert d <= 1e-6, (lev, d)
    sm.close()
    s1.close()


def test_split_smoother_solve(mg):
    """The mixed MG-CG solve at P = 32 with the split smoother (the default on
    its two finest levels) reaches 1e-10 on the FP64 residual in about as many
    iterations as the FP64 MG-CG solve."""
    import torch
    lengths, counts, P = (1.0, 1.0, 1.0), (4, 4, 4), 32
    s64 = mg.MGSolver(lengths, counts, P)
    sm = mg.MGSolver(lengths, counts, P, precision="mixed", outer_df64="all")
    assert sm.kernel_variants(sm.L)["fdm"] == 2
    b = s64.rhs(torch.tensor(inputs.gaussian(s64.num_dofs(), 43), device=s64.device))
    u64, it64, rel64, _ = s64.solve(b, tol=1e-10, use_cg=True)
    um, itm, relm, _ = sm.solve(b, tol=1e-10, use_cg=True)
    true_rel = float(torch.linalg.norm(s64.residual(um, b)) / torch.linalg.norm(b))
    assert rel64 <= 1e-10 and true_rel <= 1.01e-10, (rel64, true_rel)
    assert itm <= it64 + 2, (itm, it64)
    s64.close()
    sm.close()
