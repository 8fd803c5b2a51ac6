"""GPU test of the allocation-free coarse solve, mg_coarse_solve_noalloc.

That entry point serves callers that may not allocate device memory (a plugin
handed only its input and output buffers by a framework that owns all device
memory, or a path that cannot accept an allocation's implicit device
synchronisation): it needs no context and no workspace, and keeps its scratch
in one file-scope device array.  Here it is called through the C ABI twice in
a row and its output is compared with the existing context-based entry point
mg_coarse_solve on the same input, at the FP64 tolerance of the parity tests.
This file is collected last, and the test also passes alone in a fresh
process (its first call performs the once-per-device address lookup).
"""
import ctypes

import numpy as np
import pytest

from paper_1612_04796_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("lengths,counts", [((2.0, 1.0, 0.5), (4, 3, 5)), ((1.0, 1.0, 1.0), (32, 32, 32))])
def test_noalloc_coarse_solve_matches_context_entry_point(mg, lengths, counts):
    import torch
    lib = mg.load_library()
    s = mg.MGSolver(lengths, counts, 2)
    stream = torch.cuda.current_stream()
    N0 = s.num_dofs(0)
    for seed in (31, 32):  # two calls in a row share the static scratch
        f0 = torch.tensor(inputs.gaussian(N0, seed), device=s.device)
        ref = s.coarse_solve(f0)
        u0 = torch.full_like(f0, float("nan"))
        st = lib.mg_coarse_solve_noalloc(lengths[0], lengths[1], lengths[2], counts[0], counts[1], counts[2], 2.0,
                                         _ptr(f0), _ptr(u0), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        got = u0.cpu().numpy()
        want = ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < FP64_TOL


def test_noalloc_second_call_takes_no_device_memory(mg):
    """After a first call (which may load the module and so reserve the
    array), a further call leaves the device's free memory unchanged."""
    import torch
    lib = mg.load_library()
    lengths, counts = (1.0, 2.0, 1.0), (8, 6, 5)
    N0 = 8 * counts[0] * counts[1] * counts[2]
    f0 = torch.tensor(inputs.gaussian(N0, 33), device="cuda")
    f0 -= f0.mean()
    u0 = torch.empty_like(f0)
    stream = torch.cuda.current_stream()

    def call():
        st = lib.mg_coarse_solve_noalloc(lengths[0], lengths[1], lengths[2], counts[0], counts[1], counts[2], 2.0,
                                         _ptr(f0), _ptr(u0), ctypes.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        assert st == 0

    call()
    free0, _ = torch.cuda.mem_get_info()
    call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_the_maximum(mg):
    import torch
    lib = mg.load_library()
    buf = torch.zeros(8 * 33 * 4 * 4, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(buf)
    st = lib.mg_coarse_solve_noalloc(1.0, 1.0, 1.0, 33, 4, 4, 2.0, _ptr(buf), _ptr(out), None)
    assert st == 1  # MG_EINVAL
