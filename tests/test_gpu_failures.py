"""Failure handling on the GPU without faulting it: iteration limits end in a
status, bad arguments are rejected before any kernel runs, a NaN right-hand
side ends after maxit cycles (no hang), and the tensor-core kernel's bounded
mbarrier wait runs out on a barrier that nothing arrives on and reports it."""
import ctypes

import numpy as np
import pytest

from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small(mg):
    s = mg.MGSolver((1.0, 1.0, 1.0), (4, 4, 4), 4)
    import torch
    b = s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), 9), device=s.device))
    return s, b


def test_iteration_limit_returns_enoconv_with_partial_result(small, mg):
    s, b = small
    with pytest.raises(mg.MGError) as ei:
        s.solve(b, maxit=2, tol=1e-10)
    assert ei.value.status == 4  # MG_ENOCONV
    u, its, rel, hist = s.solve(b, maxit=2, tol=1e-10, raise_on_noconv=False)
    assert its == 2 and 1e-10 < rel < 1.0 and len(hist) == 3 and hist[2] < hist[0]


def test_bad_arguments_are_rejected(small, mg):
    import torch
    s, b = small
    lib = s.lib
    assert lib.mg_apply_sipg(s.ctx, 7, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(b.data_ptr())) == 1
    assert lib.mg_smooth(s.ctx, 0, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(b.data_ptr()), 1) == 1
    assert lib.mg_solve(s.ctx, None, ctypes.c_void_p(b.data_ptr()), 1e-10, 10, 0, None, None, None) == 1
    with pytest.raises(ValueError):
        s.apply_sipg(torch.zeros(5, dtype=torch.float64, device=s.device))


def test_nan_rhs_is_rejected_and_context_stays_usable(small, mg):
    s, b = small
    bad = b.clone()
    bad[17] = float("nan")
    with pytest.raises(mg.MGError) as ei:
        s.solve(bad, maxit=3, tol=1e-10)
    assert ei.value.status == 1  # MG_EINVAL: non-finite initial residual
    u2, its2, rel2, _ = s.solve(b, tol=1e-10)
    assert rel2 <= 1e-10


def test_tensor_core_wait_runs_out_and_context_stays_usable(mg):
    """The tensor-core smoother's mbarrier wait is bounded: with nothing ever
    arriving on the barrier (no MMA issued) the kernel gives up after its limit,
    reports the timeout in the status word and frees its tensor memory; the
    same context then solves normally."""
    import torch
    s = mg.MGSolver((1.0, 1.0, 1.0), (4, 4, 4), 8, precision="mixed", tensor_cores=True)
    assert s.fdm_tensor_cores(s.L) == 1
    flag = ctypes.c_int(-1)
    assert s.lib.mg_selftest_bounded_wait(s.ctx, s.L, ctypes.byref(flag)) == 0
    assert flag.value == 1
    b = s.rhs(torch.tensor(inputs.gaussian(s.num_dofs(), 9), device=s.device))
    u, its, rel, _ = s.solve(b, tol=1e-10, use_cg=True)
    assert rel <= 1e-10
    # a level that cannot run the kernel (FP64 context) is refused
    s64 = mg.MGSolver((1.0, 1.0, 1.0), (4, 4, 4), 4)
    assert s64.lib.mg_selftest_bounded_wait(s64.ctx, 1, ctypes.byref(flag)) == 1
    s.close()
    s64.close()
