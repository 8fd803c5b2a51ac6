"""Host logic of the native serving runtime with fake solves (no GPU): the
admission rule (mg_sched_pick) on its own, and the runtime's workers, slot
limit, memory budget, failures and latency bookkeeping driven by a Python
executor in place of the GPU solve."""
import ctypes
import threading
import time

import numpy as np
import pytest

import paper_1612_04796_gb300 as pkg
from paper_1612_04796_gb300 import _lib
from paper_1612_04796_gb300.serving import Request, Server, latency_summary, request_stream


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load_library()


def _pick(lib, policy, now, budget, used, arrival, work, footprint, max_wait=10.0):
    n = len(arrival)
    a = (ctypes.c_double * max(n, 1))(*arrival)
    w = (ctypes.c_double * max(n, 1))(*work)
    f = (ctypes.c_size_t * max(n, 1))(*footprint)
    return lib.mg_sched_pick(policy, max_wait, now, budget, used, n, ctypes.cast(a, ctypes.c_void_p),
                             ctypes.cast(w, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p))


def test_pick_fcfs_blocks_behind_the_head(lib):
    F = _lib.MG_SCHED_FCFS
    assert _pick(lib, F, 0.0, 100, 0, [0, 1, 2], [5, 1, 1], [50, 10, 10]) == 0
    assert _pick(lib, F, 0.0, 100, 60, [0, 1, 2], [5, 1, 1], [50, 10, 10]) == -1  # head does not fit
    assert _pick(lib, F, 0.0, 100, 0, [], [], []) == -1


def test_pick_smallest_fitting_then_aging(lib):
    S = _lib.MG_SCHED_SMALLEST
    arr, work, fp = [0.0, 0.1, 0.2, 0.3], [40, 10, 30, 10], [60, 50, 30, 20]
    assert _pick(lib, S, 1.0, 100, 0, arr, work, fp) == 1        # least work, earliest of the ties
    assert _pick(lib, S, 1.0, 100, 60, arr, work, fp) == 3       # 1 no longer fits: next least work that does
    assert _pick(lib, S, 1.0, 100, 90, arr, work, fp) == -1      # nothing fits
    # request 0 waited longer than max_wait: it goes first, or nobody does
    assert _pick(lib, S, 20.5, 100, 0, arr, work, fp) == 0
    assert _pick(lib, S, 20.5, 100, 50, arr, work, fp) == -1
    # two aged ones: the older first
    assert _pick(lib, S, 30.0, 100, 0, [0.0, 0.1], [9, 1], [10, 10], max_wait=5.0) == 0


def test_pick_rejects_bad_arguments(lib):
    assert _pick(lib, 7, 0.0, 1, 0, [0], [1], [1]) == -2
    assert lib.mg_sched_pick(0, 1.0, 0.0, 1, 0, 2, None, None, None) == -2


def _fake(durations, log):
    lock = threading.Lock()

    def run(req, slot):
        with lock:
            log.append(("start", req.id, slot))
        time.sleep(durations[req.id])
        with lock:
            log.append(("end", req.id, slot))
        return {"iterations": 1, "relres": 0.0}
    return run


def _admission_order(results):
    return [r.id for r in sorted(results, key=lambda r: r.t_admit)]


def _req(i, n=4, P=2, arrival=0.0, footprint=1):
    return Request(i, (1, 1, 1), (n, n, n), P, i, arrival=arrival, footprint=footprint)


def test_slots_and_budget_are_respected():
    sizes = {i: 30 if i % 2 else 50 for i in range(8)}
    reqs = [_req(i, footprint=sizes[i]) for i in range(8)]
    log = []
    srv = Server(slots=3, budget_bytes=100, executor=_fake({i: 0.02 for i in range(8)}, log))
    res = srv.serve(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert srv.max_active <= 3
    assert srv.stats().peak_used <= 100 and srv.stats().completed == 8
    # replay the log: memory in use never exceeds the budget, slots never shared
    used, busy = 0, set()
    for kind, rid, slot in log:
        if kind == "start":
            used += sizes[rid]
            assert used <= 100
            assert slot not in busy
            busy.add(slot)
        else:
            used -= sizes[rid]
            busy.discard(slot)
    # admission (the runtime's own clock, taken under its lock) is first come first served
    assert _admission_order(res) == list(range(8))
    srv.close()


def test_budget_of_one_request_serialises():
    reqs = [_req(i, footprint=60) for i in range(4)]
    srv = Server(slots=4, budget_bytes=100, executor=_fake({i: 0.01 for i in range(4)}, []))
    srv.serve(reqs, realtime=False)
    assert srv.max_active == 1
    srv.close()


def test_request_larger_than_budget_is_rejected():
    srv = Server(slots=2, budget_bytes=100, executor=_fake({0: 0.0}, []))
    with pytest.raises(ValueError):
        srv.serve([_req(0, footprint=200)], realtime=False)
    srv.close()


def test_invalid_request_is_rejected():
    srv = Server(slots=1, executor=_fake({0: 0.0}, []))
    with pytest.raises(ValueError):
        srv.serve([Request(0, (1, 1, 1), (4, 4, 4), 3, 0)], realtime=False)  # P not a power of two
    srv.close()


def test_failures_are_recorded_and_latency_summary():
    def run(req, slot):
        if req.id == 1:
            raise RuntimeError("boom")
        return {"iterations": 3, "relres": 1e-11}
    reqs = [_req(i, arrival=0.001 * i) for i in range(5)]
    srv = Server(slots=2, budget_bytes=10, executor=run)
    res = srv.serve(reqs, realtime=True)
    assert "boom" in res[1].error and all(r.error is None for i, r in enumerate(res) if i != 1)
    assert all(r.iterations == 3 for i, r in enumerate(res) if i != 1)
    assert all(r.t_arrival <= r.t_admit <= r.t_done for r in res)
    summ = latency_summary(res)
    assert summ["completed"] == 4 and summ["failed"] == 1 and summ["p99_s"] >= summ["p50_s"] >= 0
    srv.close()


def test_request_stream_shape():
    reqs = request_stream(seed=5, n_requests=512)
    assert len(reqs) == 512
    assert {r.counts[0] for r in reqs} <= {4, 8, 16, 24, 32}
    assert {r.P for r in reqs} <= {2, 4, 8, 16}
    assert all(1.0 <= r.lengths[0] <= 8.0 for r in reqs)
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and 1.5 < arr[-1] < 4.0  # ~512 / 200 per second


def test_smallest_first_admits_small_requests_first():
    """policy "smallest": with one slot held by a first request while the
    others arrive, they then run in increasing work order."""
    sizes = [16, 4, 8, 32, 4]
    reqs = [_req(i, n=n, arrival=0.1) for i, n in enumerate(sizes)] + [_req(5, n=32, arrival=0.0)]
    log = []
    gate = threading.Event()
    run = _fake({i: 0.005 for i in range(6)}, log)

    def first_waits(req, slot):  # the first request holds the slot until the others have arrived
        if req.id == 5:
            gate.wait(5.0)
        return run(req, slot)
    srv = Server(slots=1, budget_bytes=10, policy="smallest", executor=first_waits)
    t = threading.Timer(0.4, gate.set)
    t.start()
    res = srv.serve(reqs, realtime=True)
    assert _admission_order(res) == [5, 1, 4, 2, 0, 3]
    srv.close()


def test_smallest_first_skips_what_does_not_fit_and_ages():
    """A large request that does not fit does not block smaller ones; once it
    has waited longer than max_wait it goes first and is not overtaken."""
    big = _req(0, n=32, footprint=10)
    small = [_req(i, footprint=4) for i in range(1, 9)]
    log = []
    srv = Server(slots=3, budget_bytes=10, policy="smallest", max_wait=0.05,
                 executor=_fake({i: 0.03 for i in range(9)}, log))
    res = srv.serve(small[:2] + [big] + small[2:], realtime=True)
    starts = _admission_order(res)
    assert starts[0] != 0                       # small ones first while nothing aged
    i_big = starts.index(0)
    assert i_big < len(starts) - 1              # aged: admitted before the small ones are exhausted
    sizes = {0: 10}
    sizes.update({i: 4 for i in range(1, 9)})
    used, peak = 0, 0
    for kind, rid, _ in log:
        used += sizes[rid] if kind == "start" else -sizes[rid]
        peak = max(peak, used)
    assert peak <= 10
    srv.close()


def test_fill_callback_writes_the_seeded_rhs(lib):
    """The right-hand side the runtime asks for at admission is the request's
    seeded Gaussian (inputs.gaussian)."""
    from paper_1612_04796_gb300 import inputs
    srv = Server(slots=1, executor=lambda r, s: {})
    r = _req(0)
    srv._records[5] = (r, None)
    buf = np.zeros(r.dofs)
    srv._fill(5, 1, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), r.dofs)
    assert np.array_equal(buf, inputs.gaussian(r.dofs, r.seed))
    srv.close()


def test_unknown_policy_is_rejected():
    with pytest.raises(ValueError):
        Server(slots=1, policy="lifo", executor=lambda r, s: {})


def test_poll_wait_and_ticket_release(lib):
    """mg_poll says not ready while a request runs, hands the result out
    once, and forgets the ticket afterwards."""
    gate = threading.Event()

    def run(req, slot):
        gate.wait(5.0)
        return {"iterations": 7, "relres": 0.5}
    srv = Server(slots=1, executor=run)
    q = srv._request(_req(0), 1, None)
    srv._records[1] = (_req(0), None)
    t = ctypes.c_longlong()
    assert lib.mg_submit(srv.handle, ctypes.byref(q), ctypes.byref(t)) == 0
    out = _lib.MgResult()
    assert lib.mg_poll(srv.handle, t.value, ctypes.byref(out)) == _lib.MG_ENOTREADY
    assert lib.mg_wait(srv.handle, t.value, 0.01, ctypes.byref(out)) == _lib.MG_ENOTREADY
    gate.set()
    assert lib.mg_wait(srv.handle, t.value, -1.0, ctypes.byref(out)) == 0
    assert out.status == 0 and out.iterations == 7 and out.relres == 0.5 and out.slot == 0
    assert lib.mg_poll(srv.handle, t.value, ctypes.byref(out)) == _lib.MG_EINVAL
    assert lib.mg_poll(srv.handle, 12345, ctypes.byref(out)) == _lib.MG_EINVAL
    srv.close()


def test_destroy_finishes_submitted_work(lib):
    done = []

    def run(req, slot):
        time.sleep(0.01)
        done.append(req.id)
        return {}
    srv = Server(slots=2, executor=run)
    for i in range(6):
        srv._records[i + 1] = (_req(i), None)
        q = srv._request(_req(i), i + 1, None)
        t = ctypes.c_longlong()
        assert lib.mg_submit(srv.handle, ctypes.byref(q), ctypes.byref(t)) == 0
    srv.close()
    assert sorted(done) == list(range(6))


def test_library_footprint_is_host_only(lib):
    srv = Server(slots=1, executor=lambda r, s: {})
    big, small = Request(0, (1, 1, 1), (8, 8, 8), 8, 0), Request(1, (1, 1, 1), (4, 4, 4), 2, 0)
    fb, fs = srv.footprint(big), srv.footprint(small)
    assert fb > 3 * 8 * big.dofs and fs > 3 * 8 * small.dofs and fb > fs
    srv.close()


def test_server_options_are_validated(lib):
    """mg_server_create rejects bad options on the host (custom executor: no
    CUDA call): slots, policy, batch size."""
    fn = _lib.EXECUTE_FN(lambda *a: 0)
    for field, value in (("slots", 0), ("slots", 257), ("policy", 2), ("batch_max", 0), ("batch_max", 17),
                         ("maxit", 0), ("max_wait", -1.0)):
        o = _lib.MgServerOpts()
        lib.mg_server_default_opts(ctypes.byref(o))
        o.execute = fn
        setattr(o, field, value)
        h = ctypes.c_void_p()
        assert lib.mg_server_create(ctypes.byref(o), ctypes.byref(h)) == _lib.MG_EINVAL, field
    o = _lib.MgServerOpts()
    lib.mg_server_default_opts(ctypes.byref(o))
    assert (o.slots, o.policy, o.maxit, o.use_cg, o.batch_max, o.batch_dofs) == (8, 0, 400, 1, 16, 1 << 20)


def test_small_request_stream_shape():
    """The saturated small-request stream: sizes, orders and arrival rate as asked."""
    reqs = request_stream(seed=5, n_requests=512, rate=5000.0, sizes=(4, 8), orders=(2, 4, 8))
    assert {r.counts[0] for r in reqs} <= {4, 8} and {r.P for r in reqs} <= {2, 4, 8}
    assert max(r.dofs for r in reqs) <= 8 ** 3 * 9 ** 3
    assert 0.05 < reqs[-1].arrival < 0.2  # ~512 / 5000 per second
