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
    srv = Server(slots=4)
    srv.scheduler.budget = srv.footprint(reqs[0])
    res = srv.serve(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert srv.max_active == 1
