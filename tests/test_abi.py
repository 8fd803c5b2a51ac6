"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/mgdg.h declares, and its host-only logic (argument validation, level
sizes, overlap layers, workspace sizing, not-ready errors) behaves.  No
compute call is made: there is no GPU here."""
import ctypes
import json
import os

import pytest

import paper_1612_04796_gb300 as pkg
from paper_1612_04796_gb300._lib import MgOpts

HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load_library()


def test_exports_every_declared_symbol(lib):
    names = pkg.header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def _setup(lib, P=4, counts=(4, 4, 4), overlap=1, lengths=(1.0, 1.0, 1.0), **kw):
    opts = MgOpts()
    lib.mg_default_opts(ctypes.byref(opts))
    for k, v in kw.items():
        setattr(opts, k, v)
    ctx = ctypes.c_void_p()
    st = lib.mg_setup(lengths[0], lengths[1], lengths[2], counts[0], counts[1], counts[2], P, 2.0, overlap,
                      ctypes.byref(opts), ctypes.byref(ctx))
    return st, ctx


def test_defaults(lib):
    o = MgOpts()
    lib.mg_default_opts(ctypes.byref(o))
    assert (o.ns_pre, o.ns_post, o.ns_growth, o.precision, o.overlap_mode, o.weight_profile) == (1, 1, 1, 0, 0, 0)


@pytest.mark.parametrize("bad", [dict(P=3), dict(P=1), dict(P=64), dict(counts=(2, 4, 4)), dict(counts=(4, 4, 513)),
                                 dict(overlap=-1), dict(lengths=(0.0, 1.0, 1.0)), dict(ns_pre=0, ns_post=0),
                                 dict(precision=7), dict(overlap_mode=1, overlap_frac=0.75),
                                 dict(weight_delta=4), dict(weight_delta=3), dict(overlap_mode=2, weight_delta=1),
                                 dict(autotune=2), dict(precision=1, outer_df64=3),
                                 dict(precision=1, fdm_tensor_cores=3)])
def test_rejects_bad_arguments(lib, bad):
    st, ctx = _setup(lib, **bad)
    assert st == 1 and not ctx.value


@pytest.mark.parametrize("P", [2, 4, 8, 16, 32])
def test_levels_and_sizes(lib, P):
    st, ctx = _setup(lib, P=P, counts=(3, 4, 5), overlap=4)
    assert st == 0
    L = P.bit_length() - 1
    assert lib.mg_num_levels(ctx) == L + 1
    for l in range(L + 1):
        assert lib.mg_num_dofs(ctx, l) == 60 * (2 ** l + 1) ** 3
        if l >= 1:
            assert lib.mg_level_layers(ctx, l) == min(4, 2 ** (l - 1) + 1)
    assert lib.mg_num_dofs(ctx, L + 1) == -1
    sz = ctypes.c_size_t()
    assert lib.mg_workspace_size(ctx, ctypes.byref(sz)) == 0
    assert sz.value > 8 * 60 * (P + 1) ** 3 * 10
    lib.mg_destroy(ctx)


def test_width_overlap_reproduces_table1_layers(lib):
    table = json.load(open(os.path.join(HERE, "golden", "table1_gll.json")))
    for row in table["rows"]:
        if not row["overlap"].startswith("delta_O"):
            continue
        frac = float(row["overlap"].split("=")[1])
        st, ctx = _setup(lib, P=32, overlap_mode=1, overlap_frac=frac)
        assert st == 0
        got = [lib.mg_level_layers(ctx, l) for l in range(1, 6)]
        assert got == row["n_o"], (frac, got)
        lib.mg_destroy(ctx)


def test_calls_before_binding_are_not_ready(lib):
    st, ctx = _setup(lib)
    assert st == 0
    dummy = ctypes.c_void_p(256)
    assert lib.mg_apply_sipg(ctx, 2, dummy, dummy) == 5
    assert lib.mg_vcycle(ctx, dummy, dummy) == 5
    assert b"not bound" in lib.mg_last_error(ctx)
    # misaligned / too small workspace is rejected before any CUDA call
    assert lib.mg_bind_workspace(ctx, ctypes.c_void_p(257), ctypes.c_size_t(1 << 40)) == 1
    assert lib.mg_bind_workspace(ctx, ctypes.c_void_p(256), ctypes.c_size_t(16)) == 2
    lib.mg_destroy(ctx)


@pytest.mark.parametrize("ar", [1, 3, 8, 12, 48])
@pytest.mark.parametrize("P", [4, 16])
def test_max_overlap_layers_per_direction(lib, ar, P):
    """MG_OVERLAP_MAX: N_O of every level and direction equals the oracle's
    count for delta_O,i = min(0.08 max_j dx_j, dx_i) (Table 2)."""
    import math

    from oracle.schwarz import max_width_layers
    from oracle.multigrid import max_overlap_widths
    from oracle.sipg import Mesh
    lengths = (2 * math.pi * ar, 2 * math.pi * math.ceil(ar / 2), 2 * math.pi)
    st, ctx = _setup(lib, P=P, counts=(8, 8, 8), lengths=lengths, overlap_mode=2, overlap_frac=0.08)
    assert st == 0
    deltas = max_overlap_widths(Mesh(lengths, (8, 8, 8)), 0.08)
    for l in range(1, P.bit_length()):
        got = [lib.mg_level_layers_dir(ctx, l, d) for d in range(3)]
        assert got == [max_width_layers(2 ** l, dd) for dd in deltas], (l, got)
        assert lib.mg_level_layers(ctx, l) == got[0]
    assert lib.mg_level_layers_dir(ctx, 1, 3) == -1
    lib.mg_destroy(ctx)


def test_max_overlap_rejections(lib):
    import math
    lengths = (2 * math.pi * 48, 2 * math.pi * 24, 2 * math.pi)
    # whole-element strips in z with only three elements there
    st, ctx = _setup(lib, P=4, counts=(4, 4, 3), lengths=lengths, overlap_mode=2, overlap_frac=0.08)
    assert st == 1 and not ctx.value
    st, ctx = _setup(lib, P=4, counts=(4, 4, 4), lengths=lengths, overlap_mode=2, overlap_frac=1.5)
    assert st == 1 and not ctx.value
    st, ctx = _setup(lib, P=4, counts=(4, 4, 4), lengths=lengths, overlap_mode=3, overlap_frac=0.08)
    assert st == 1 and not ctx.value


def test_batch_solve_argument_checks(lib):
    """mg_solve_batch rejects bad arguments on the host (no CUDA call): no
    contexts, a count out of range, a context without workspace."""
    st, ctx = _setup(lib)
    assert st == 0
    P = ctypes.c_void_p
    ctxs = (P * 1)(ctx.value)
    vec = (P * 1)(P(256))
    its = (ctypes.c_int * 1)()
    rel = (ctypes.c_double * 1)()
    sts = (ctypes.c_int * 1)()
    args = (ctypes.cast(vec, P), ctypes.cast(vec, P), 1e-10, 10, ctypes.cast(its, P), ctypes.cast(rel, P),
            ctypes.cast(sts, P))
    assert lib.mg_solve_batch(None, 1, *args) == 1                       # MG_EINVAL
    assert lib.mg_solve_batch(ctypes.cast(ctxs, P), 0, *args) == 1
    assert lib.mg_solve_batch(ctypes.cast(ctxs, P), 17, *args) == 1
    assert lib.mg_solve_batch(ctypes.cast(ctxs, P), 1, *args) == 5       # MG_ENOTREADY: not bound
    assert lib.mg_batch_launches(ctx) == 0
    lib.mg_destroy(ctx)


def test_weight_delta_readings_accepted(lib):
    """Node-based half-width readings in both overlap modes, the strip reading
    only for the geometric overlap."""
    for mode, delta in ((0, 1), (0, 2), (1, 1), (1, 2), (1, 3), (2, 0)):
        st, ctx = _setup(lib, P=16, overlap=2, overlap_mode=mode, overlap_frac=0.08, weight_delta=delta)
        assert st == 0, (mode, delta)
        lib.mg_destroy(ctx)


def test_kernel_variant_query(lib):
    st, ctx = _setup(lib, P=8, counts=(4, 4, 4), autotune=1)
    assert st == 0
    assert lib.mg_level_kernel_variant(ctx, 0, 0) == -1
    assert lib.mg_level_kernel_variant(ctx, 3, 3) == -1
    assert lib.mg_level_kernel_variant(ctx, 4, 0) == -1
    assert lib.mg_level_kernel_variant(ctx, 3, 0) == 0  # before binding: the defaults
    lib.mg_destroy(ctx)


def _setup_graded(lib, widths, P=4, overlap=1, **kw):
    import numpy as np
    opts = MgOpts()
    lib.mg_default_opts(ctypes.byref(opts))
    for k, v in kw.items():
        setattr(opts, k, v)
    ws = [np.ascontiguousarray(w, dtype=np.float64) for w in widths]
    ctx = ctypes.c_void_p()
    st = lib.mg_setup_graded(*(w.ctypes.data_as(ctypes.c_void_p) for w in ws), len(ws[0]), len(ws[1]), len(ws[2]),
                             P, 2.0, overlap, ctypes.byref(opts), ctypes.byref(ctx))
    return st, ctx


def test_graded_setup_host_validation(lib):
    """mg_setup_graded: valid widths give a context flagged as graded whose
    workspace holds the per-line tables (more than the uniform context of the
    same counts); invalid widths, sizes and unsupported options are refused
    before any CUDA call."""
    w = [[0.2, 0.5, 0.3], [0.4, 0.4, 0.2, 0.5], [1.0, 2.0, 0.5]]
    st, ctx = _setup_graded(lib, w, P=8)
    assert st == 0 and lib.mg_is_graded(ctx) == 1
    gsize = ctypes.c_size_t()
    assert lib.mg_workspace_size(ctx, ctypes.byref(gsize)) == 0
    assert lib.mg_num_dofs(ctx, 3) == 36 * 729
    st2, uctx = _setup(lib, P=8, counts=(3, 4, 3))
    usize = ctypes.c_size_t()
    assert st2 == 0 and lib.mg_is_graded(uctx) == 0
    lib.mg_workspace_size(uctx, ctypes.byref(usize))
    assert gsize.value > usize.value
    buf = (ctypes.c_double * 16)()
    cnt = ctypes.c_int()
    assert lib.mg_get_line_table(ctx, 3, 0, 0, 0, buf, 16, ctypes.byref(cnt)) == 5  # MG_ENOTREADY
    lib.mg_destroy(ctx)
    lib.mg_destroy(uctx)
    bad = [
        ([[0.2, -0.5, 0.3], w[1], w[2]], {}),
        ([[0.2, float("nan"), 0.3], w[1], w[2]], {}),
        ([[0.5, 0.5], w[1], w[2]], {}),
        ([[0.01] * 257, w[1], w[2]], {}),
        (w, {"precision": 2}),
        (w, {"overlap_mode": 1}),
        (w, {"precision": 1, "fdm_tensor_cores": 1}),
        (w, {"autotune": 1}),
    ]
    for widths, kw in bad:
        st, c = _setup_graded(lib, widths, **kw)
        assert st == 1 and not c.value, (widths if not kw else kw)


def test_bench_graded_workload_widths():
    """The graded bench workload: smooth periodic widths summing to the box
    length, largest / smallest at most (1 + 0.6) / (1 - 0.6) = 4, neighbouring
    widths within a factor 1.35, accepted by mg_setup_graded."""
    import numpy as np

    import bench
    W = bench.WORKLOADS["graded16_p8"]
    assert len(W["widths"]) == 3
    for d, w in enumerate(W["widths"]):
        w = np.asarray(w)
        assert len(w) == W["elements"][d]
        assert abs(w.sum() - W["lengths"][d]) < 1e-14
        assert w.max() / w.min() <= 4.0 + 1e-12
        assert np.max(np.maximum(w / np.roll(w, 1), np.roll(w, 1) / w)) < 1.35
    lib = pkg.load_library()
    st, ctx = _setup_graded(lib, W["widths"], P=W["P"], overlap=W["overlap_layers"])
    assert st == 0
    lib.mg_destroy(ctx)
