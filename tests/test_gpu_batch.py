"""Batched MG-CG (mg_solve_batch): problems of different boxes, meshes and
aspect ratios advanced together give bitwise the results of their own
solves, with fewer launches than the solves one by one."""
import numpy as np
import pytest

from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu

# (lengths, counts, P): uneven meshes of one order; 4^3 and 5^3 elements take
# the direction-split operator, the larger ones the element-block operator
SHAPES = [((1.0, 1.0, 1.0), (4, 4, 4)), ((3.0, 1.0, 1.0), (8, 8, 8)), ((1.0, 2.0, 1.0), (5, 6, 7)),
          ((6.5, 1.0, 1.0), (4, 4, 4)), ((1.0, 1.0, 1.0), (9, 8, 8))]


def _problems(mg, P, precision, outer_df64, overlap=1):
    import torch
    out = []
    for i, (L, n) in enumerate(SHAPES):
        s = mg.MGSolver(L, n, P, overlap=overlap, precision=precision, outer_df64=outer_df64)
        b = s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), 300 + i), device="cuda"))
        out.append((s, b))
    return out


@pytest.mark.parametrize("P,precision,outer_df64,overlap", [(4, "mixed", True, 1), (8, "mixed", False, 2),
                                                            (2, "fp64", False, 1), (4, "df64", False, 1)])
def test_batch_equals_individual_solves(mg, P, precision, outer_df64, overlap):
    import torch
    probs = _problems(mg, P, precision, outer_df64, overlap)
    ref = []
    for s, b in probs:
        u, its, rel, _ = s.solve(b, tol=1e-10, use_cg=True, maxit=200)
        ref.append((u.clone(), its, rel))
    n0 = [s.kernel_launches() for s, _ in probs]
    us, its, rels, sts = mg.solve_batch([s for s, _ in probs], [b for _, b in probs], tol=1e-10, maxit=200)
    torch.cuda.synchronize()
    for (u_ref, it_ref, rel_ref), u, it, rel, st in zip(ref, us, its, rels, sts):
        assert st == 0
        assert it == it_ref and rel == rel_ref
        assert torch.equal(u, u_ref)
    for s, _ in probs:
        s.close()


def test_batch_mixed_orders_and_limits(mg):
    """Problems of different orders in one batch (no launches merge across
    orders, the results are still each problem's own); a problem that hits
    maxit reports MG_ENOCONV without stopping the others; argument checks."""
    import torch
    from paper_1612_04796_gb300 import _lib
    a = mg.MGSolver((1.0, 1.0, 1.0), (4, 4, 4), 4, precision="mixed", outer_df64=True)
    b = mg.MGSolver((2.0, 1.0, 1.0), (5, 5, 5), 8, precision="mixed", outer_df64=True)
    fa = a.rhs(torch.tensor(inputs.gaussian(a.num_dofs(), 1), device="cuda"))
    fb = b.rhs(torch.tensor(inputs.gaussian(b.num_dofs(), 2), device="cuda"))
    ua, ita, _, _ = a.solve(fa, tol=1e-10, use_cg=True)
    ub, itb, _, _ = b.solve(fb, tol=1e-10, use_cg=True)
    us, its, rels, sts = mg.solve_batch([a, b], [fa, fb], tol=1e-10)
    assert sts == [0, 0] and its == [ita, itb]
    assert torch.equal(us[0], ua) and torch.equal(us[1], ub)
    us, its, rels, sts = mg.solve_batch([a, b], [fa, fb], tol=1e-10, maxit=3)
    assert sts == [_lib.MG_ENOCONV, _lib.MG_ENOCONV] and its == [3, 3]
    with pytest.raises(mg.MGError):
        mg.solve_batch([a, a], [fa, fa])
    a.close()
    b.close()
