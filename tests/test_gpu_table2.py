"""The anisotropic study of Section 4.2 (Table 2 / Fig. 6, whose data the
source does not contain): 8^3 elements, P = 16, domain
(0, AR) x (0, ceil(AR/2)) x (0, 1) (scale-free version of the paper's 2 pi
boxes), MG-CG with delta_O = 0.08 dx_i on every level ("0.08 rel"), fixed
V(1,1) versus the variable V-cycle N_s,l = (1,1) x 3^(L-l).

Checked against the paper's statements that hold here: at AR = 1 both behave
like Table 1 (P = 16, n10 about 5); the fixed cycle keeps converging but
slows strongly with AR (rho from about 0.01 to about 0.6 at AR = 16, "two
orders of magnitude"); the variable cycle is at least as good up to AR = 12.
Not reproduced: beyond AR = 12 the variable cycle falls behind the fixed one
here, while the paper reports it stays superior; the paper's robust
"0.08 max" strategy needs a different overlap per direction, not built."""
import math

import pytest

from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu

ARS = (1, 2, 4, 8, 12, 16, 24, 32, 48)


def _n10(mg, ar, growth, use_cg=True):
    import torch
    s = mg.MGSolver((float(ar), float(math.ceil(ar / 2)), 1.0), (8, 8, 8), 16, overlap_mode="width",
                    overlap_frac=0.08, ns_growth=growth)
    N = s.num_dofs()
    u0 = torch.tensor(inputs.uniform_guess(N, 1), device=s.device)
    f = torch.zeros(N, dtype=torch.float64, device=s.device)
    _, its, _, hist = s.solve(f, u0, tol=1e-10, maxit=200, use_cg=use_cg, raise_on_noconv=False)
    s.close()
    rho = (hist[-1] / hist[0]) ** (1.0 / (len(hist) - 1))
    return math.ceil(-10.0 / math.log10(rho)), rho


def test_variable_cycle_is_robust_up_to_ar12(mg):
    lines = ["| AR | n10 fixed V(1,1) | rho fixed | n10 variable | rho variable |", "|---|---|---|---|---|"]
    fix, var = {}, {}
    for ar in ARS:
        nf, rf = _n10(mg, ar, 1)
        nv, rv = _n10(mg, ar, 3)
        fix[ar], var[ar] = nf, nv
        lines.append("| %d | %d | %.3g | %d | %.3g |" % (ar, nf, rf, nv, rv))
    print("\n" + "\n".join(lines))
    assert fix[1] <= 6 and var[1] <= fix[1]                       # Table 1 rows 3-4, P = 16: n10 = 5
    assert all(fix[a] <= fix[b] for a, b in zip(ARS, ARS[1:]))    # monotone degradation with AR
    assert fix[16] >= 5 * fix[1]                                   # strongly slowed by AR = 16
    assert all(var[ar] <= fix[ar] for ar in ARS if ar <= 12)       # variable cycle helps up to AR = 12
