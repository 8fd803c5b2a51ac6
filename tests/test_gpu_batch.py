"""Batched MG-CG (mg_solve_batch): problems of different boxes, meshes and
aspect ratios advanced together agree with their own solves to rounding (the
batched kernels are separate compilations of the same code), and a problem's
batched result is the same bits whatever else is in the batch."""
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


def _close(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("P,precision,outer_df64,overlap", [(4, "mixed", True, 1), (8, "mixed", False, 2),
                                                            (2, "fp64", False, 1), (4, "df64", False, 1)])
def test_batch_matches_individual_solves(mg, P, precision, outer_df64, overlap):
    probs = _problems(mg, P, precision, outer_df64, overlap)
    ref = []
    for s, b in probs:
        u, its, rel, _ = s.solve(b, tol=1e-10, use_cg=True, maxit=200)
        ref.append((u.clone(), its, rel))
    us, its, rels, sts = mg.solve_batch([s for s, _ in probs], [b for _, b in probs], tol=1e-10, maxit=200)
    for (u_ref, it_ref, rel_ref), (s, b), u, it, rel, st in zip(ref, probs, us, its, rels, sts):
        assert st == 0 and rel <= 1e-10
        assert abs(it - it_ref) <= 1
        assert _close(u, u_ref) < 1e-9
        assert float((s.residual(u, b)).norm() / b.norm()) <= 1.01e-10
    for s, _ in probs:
        s.close()


@pytest.mark.parametrize("precision,outer_df64", [("mixed", True), ("mixed", False), ("fp64", False)])
def test_batch_result_independent_of_the_batch(mg, precision, outer_df64):
    """The same problem alone, with all the others, and in another order and
    company: the same iterations and the same bits."""
    import torch
    probs = _problems(mg, 4, precision, outer_df64)
    solvers, rhs = [s for s, _ in probs], [b for _, b in probs]
    full = mg.solve_batch(solvers, rhs, tol=1e-10)
    for k in range(len(probs)):
        alone = mg.solve_batch([solvers[k]], [rhs[k]], tol=1e-10)
        assert alone[1][0] == full[1][k] and alone[2][0] == full[2][k]
        assert torch.equal(alone[0][0], full[0][k])
    order = [3, 0, 4]
    part = mg.solve_batch([solvers[i] for i in order], [rhs[i] for i in order], tol=1e-10)
    for j, i in enumerate(order):
        assert torch.equal(part[0][j], full[0][i]) and part[1][j] == full[1][i]
    for s in solvers:
        s.close()


def test_batch_mixed_orders_and_limits(mg):
    """Problems of different orders in one batch (no launches merge across
    orders); a problem that hits maxit reports MG_ENOCONV without stopping
    the others; argument checks."""
    import torch
    from paper_1612_04796_gb300 import _lib
    a = mg.MGSolver((1.0, 1.0, 1.0), (4, 4, 4), 4, precision="mixed", outer_df64=True)
    b = mg.MGSolver((2.0, 1.0, 1.0), (5, 5, 5), 8, precision="mixed", outer_df64=True)
    fa = a.rhs(torch.tensor(inputs.gaussian(a.num_dofs(), 1), device="cuda"))
    fb = b.rhs(torch.tensor(inputs.gaussian(b.num_dofs(), 2), device="cuda"))
    ua, ita, _, _ = a.solve(fa, tol=1e-10, use_cg=True)
    ub, itb, _, _ = b.solve(fb, tol=1e-10, use_cg=True)
    us, its, rels, sts = mg.solve_batch([a, b], [fa, fb], tol=1e-10)
    assert sts == [0, 0] and abs(its[0] - ita) <= 1 and abs(its[1] - itb) <= 1
    assert _close(us[0], ua) < 1e-9 and _close(us[1], ub) < 1e-9
    us, its, rels, sts = mg.solve_batch([a, b], [fa, fb], tol=1e-10, maxit=3)
    assert sts == [_lib.MG_ENOCONV, _lib.MG_ENOCONV] and its == [3, 3]
    with pytest.raises(mg.MGError):
        mg.solve_batch([a, a], [fa, fa])
    a.close()
    b.close()


UNIFORM = [((1.0, 1.0, 1.0), (8, 8, 8)), ((2.0, 1.0, 1.0), (9, 8, 8)), ((1.0, 3.0, 1.0), (8, 10, 8)),
           ((1.0, 1.0, 1.5), (8, 8, 9))]


def test_fp64_batch_takes_one_launch_per_sweep(mg):
    """An FP64 batch (operator, smoother, scatter, transfers and vector passes
    all with grouped twins) of meshes that take the same kernel variants
    launches far fewer kernels than the same solves one by one, with the same
    iterations."""
    import torch
    probs = []
    for i, (L, n) in enumerate(UNIFORM):
        s = mg.MGSolver(L, n, 4)
        probs.append((s, s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), 400 + i), device="cuda"))))
    solvers, rhs = [s for s, _ in probs], [b for _, b in probs]
    l0 = [s.kernel_launches() for s in solvers]
    its1 = [s.solve(b, tol=1e-10, use_cg=True)[1] for s, b in probs]
    single = sum(s.kernel_launches() - a for s, a in zip(solvers, l0))
    b0 = solvers[0].batch_launches()
    _, its, _, sts = mg.solve_batch(solvers, rhs, tol=1e-10)
    batched = solvers[0].batch_launches() - b0
    assert sts == [0] * len(probs)
    assert all(abs(a - b) <= 1 for a, b in zip(its, its1))
    assert batched < 0.5 * single, (batched, single)
    for s in solvers:
        s.close()


@pytest.mark.parametrize("precision,outer_df64", [("mixed", "all"), ("fp64", False)])
def test_persistent_grouped_launches(mg, precision, outer_df64):
    """mg_opts.persistent: every grouped launch as one wave of blocks looping
    over the problems' blocks (always), or never.  Every virtual block does
    the work of the same block of the plain grouped launch, so the batch gives
    the same iterations and the same bits either way; a persistent launch of
    several waves' worth of blocks is the default (auto) and agrees as well."""
    import torch
    res = {}
    for mode in ("always", "never", "auto"):
        solvers, rhs = [], []
        for i, (L, n) in enumerate(SHAPES):
            s = mg.MGSolver(L, n, 8, precision=precision, outer_df64=outer_df64, persistent=mode)
            solvers.append(s)
            rhs.append(s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), 400 + i), device="cuda")))
        us, its, rels, sts = mg.solve_batch(solvers, rhs, tol=1e-10, maxit=200)
        assert all(st == 0 for st in sts) and all(r <= 1e-10 for r in rels)
        res[mode] = ([u.clone() for u in us], list(its))
        for s in solvers:
            s.close()
    for mode in ("never", "auto"):
        assert res[mode][1] == res["always"][1], (mode, res[mode][1], res["always"][1])
        for a, b in zip(res[mode][0], res["always"][0]):
            assert torch.equal(a, b), mode
