"""Serving on the GPU: requests solved concurrently (continuous batching,
one stream per slot) give the same result as the same request solved alone,
and the solves really overlapped."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _requests():
    from paper_1612_04796_gb300.serving import Request
    shapes = [((1.0, 1.0, 1.0), 4, 2), ((2.5, 1.0, 1.0), 3, 4), ((1.0, 1.0, 1.0), 5, 2), ((3.0, 1.0, 1.0), 4, 4),
              ((1.5, 1.0, 1.0), 3, 8), ((1.0, 1.0, 1.0), 6, 2)]
    return [Request(i, L, (n, n, n), P, seed=100 + i) for i, (L, n, P) in enumerate(shapes)]


def test_same_result_alone_and_in_the_mix(mg):
    from paper_1612_04796_gb300.serving import Server
    alone = Server(slots=1)
    ref = alone.serve(_requests(), realtime=False)
    mix = Server(slots=4)
    got = mix.serve(_requests(), realtime=False)
    assert mix.max_active > 1
    for a, b in zip(ref, got):
        assert a.error is None and b.error is None
        assert a.iterations == b.iterations
        assert b.relres <= 1e-10
        np.testing.assert_array_equal(a.u, b.u)  # deterministic kernels: bitwise identical


def test_memory_budget_limits_concurrency(mg):
    """With a budget of one request's footprint, equal-sized requests run one
    at a time even with free slots."""
    from paper_1612_04796_gb300.serving import Request, Server
    reqs = [Request(i, (1.0, 1.0, 1.0), (4, 4, 4), 4, seed=200 + i) for i in range(4)]
    probe = Server(slots=1)
    fp = probe.footprint(reqs[0])
    probe.close()
    srv = Server(slots=4, budget_bytes=fp)
    res = srv.serve(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert srv.max_active == 1
    assert srv.stats().peak_used == fp
    srv.close()


def test_served_solution_equals_a_direct_solve(mg):
    """The runtime's path (right-hand side drawn at admission, copied in,
    assembled by mg_rhs, solved from zero, copied out) gives the bits of the
    same solve made directly: a small request takes the batched path
    (mg_solve_batch), a large one mg_solve; both agree with mg_solve to
    rounding."""
    import torch
    from paper_1612_04796_gb300 import inputs
    from paper_1612_04796_gb300.serving import Request, Server
    small = Request(0, (2.0, 1.0, 1.0), (5, 5, 5), 4, seed=77)
    large = Request(1, (1.0, 1.0, 1.0), (12, 12, 12), 8, seed=78)   # 373,248 DOFs > batch_dofs below
    srv = Server(slots=2, batch_dofs=200000)
    res = srv.serve([small, large], realtime=False)
    srv.close()
    for req, r in zip((small, large), res):
        assert r.error is None and r.relres <= 1e-10
        s = mg.MGSolver(req.lengths, req.counts, req.P, overlap=req.overlap, precision="mixed",
                        outer_df64=srv.outer_df64)
        b = s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), req.seed), device="cuda"))
        u, its, rel, _ = s.solve(b, tol=req.tol, use_cg=True, maxit=400)
        if req is small:
            ub, itb, relb, _ = mg.solve_batch([s], [b], tol=req.tol, maxit=400)
            assert itb[0] == r.iterations and relb[0] == r.relres
            np.testing.assert_array_equal(ub[0].cpu().numpy(), r.u)
            assert abs(its - r.iterations) <= 1
            assert np.max(np.abs(u.cpu().numpy() - r.u)) <= 1e-9 * np.max(np.abs(r.u))
        else:
            assert its == r.iterations and rel == r.relres
            np.testing.assert_array_equal(u.cpu().numpy(), r.u)
        s.close()


def test_fp64_standalone_server(mg):
    """Solver options reach every request: an FP64 standalone-V-cycle server
    reproduces the 12 cycles of the 16^3-element, P = 8 problem class on a
    smaller mesh of the same order (Table 1 row 1: about 11-12 cycles)."""
    from paper_1612_04796_gb300.serving import Request, Server
    srv = Server(slots=1, precision="fp64", use_cg=False)
    res = srv.serve([Request(0, (1.0, 1.0, 1.0), (6, 6, 6), 8, seed=5)], realtime=False)[0]
    srv.close()
    assert res.error is None and res.relres <= 1e-10
    assert 10 <= res.iterations <= 13


def test_batched_admission_matches_unbatched(mg):
    """Small requests of one order queued behind a busy slot are admitted
    together and solved as one batch (mg_solve_batch); every result is
    bitwise the one of the same server with groups of one."""
    from paper_1612_04796_gb300.serving import Request, Server
    reqs = [Request(i, (1.0 + 0.5 * i, 1.0, 1.0), (4 + i % 3, 4, 5), 4, seed=400 + i) for i in range(7)]
    plain = Server(slots=1, batch_max=1)
    ref = plain.serve(reqs, realtime=False)
    plain.close()
    batched = Server(slots=1, batch_max=8)
    got = batched.serve(reqs, realtime=False)
    batched.close()
    assert max(r.batch for r in got) > 1 and all(r.batch == 1 for r in ref)
    for a, b in zip(ref, got):
        assert a.error is None and b.error is None
        assert a.iterations == b.iterations and a.relres == b.relres
        np.testing.assert_array_equal(a.u, b.u)
