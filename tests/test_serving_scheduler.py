"""Host logic of the serving loop with fake solves (no GPU): first-come
first-served admission under a slot limit and a memory budget."""
import threading
import time

import pytest

from paper_1612_04796_gb300.serving import Request, Scheduler, latency_summary, request_stream


def _fake(durations, log):
    lock = threading.Lock()
    state = {"active": 0, "used": 0}

    def run(req, slot):
        with lock:
            log.append(("start", req.id, slot))
        time.sleep(durations[req.id])
        with lock:
            log.append(("end", req.id, slot))
        return {"iterations": 1, "relres": 0.0}
    return run


def test_slots_and_budget_are_respected():
    reqs = [Request(i, (1, 1, 1), (4, 4, 4), 2, i, arrival=0.0) for i in range(8)]
    log = []
    sizes = {i: 30 if i % 2 else 50 for i in range(8)}
    sched = Scheduler(_fake({i: 0.02 for i in range(8)}, log), lambda r: sizes[r.id], slots=3, budget_bytes=100)
    res = sched.serve(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert sched.max_active <= 3
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
    # admission is first come first served
    starts = [rid for kind, rid, _ in log if kind == "start"]
    assert starts == sorted(starts)


def test_budget_of_one_request_serialises():
    reqs = [Request(i, (1, 1, 1), (4, 4, 4), 2, i) for i in range(4)]
    sched = Scheduler(_fake({i: 0.01 for i in range(4)}, []), lambda r: 60, slots=4, budget_bytes=100)
    sched.serve(reqs, realtime=False)
    assert sched.max_active == 1


def test_request_larger_than_budget_is_rejected():
    sched = Scheduler(_fake({0: 0.0}, []), lambda r: 200, slots=2, budget_bytes=100)
    with pytest.raises(ValueError):
        sched.serve([Request(0, (1, 1, 1), (4, 4, 4), 2, 0)], realtime=False)


def test_failures_are_recorded_and_latency_summary():
    def run(req, slot):
        if req.id == 1:
            raise RuntimeError("boom")
        return {"iterations": 3, "relres": 1e-11}
    reqs = [Request(i, (1, 1, 1), (4, 4, 4), 2, i, arrival=0.001 * i) for i in range(5)]
    res = Scheduler(run, lambda r: 1, slots=2, budget_bytes=10).serve(reqs, realtime=True)
    assert res[1].error is not None and all(r.error is None for i, r in enumerate(res) if i != 1)
    summ = latency_summary(res)
    assert summ["completed"] == 4 and summ["failed"] == 1 and summ["p99_s"] >= summ["p50_s"] >= 0


def test_request_stream_shape():
    reqs = request_stream(seed=5, n_requests=512)
    assert len(reqs) == 512
    assert {r.counts[0] for r in reqs} <= {4, 8, 16, 24, 32}
    assert {r.P for r in reqs} <= {2, 4, 8, 16}
    assert all(1.0 <= r.lengths[0] <= 8.0 for r in reqs)
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and 1.5 < arr[-1] < 4.0  # ~512 / 200 per second


def test_smallest_first_admits_small_requests_first():
    """policy "smallest": with one slot and everything arrived, the requests
    run in increasing work order."""
    reqs = [Request(i, (1, 1, 1), (n, n, n), 2, i, arrival=0.0) for i, n in enumerate([16, 4, 8, 32, 4])]
    log = []
    sched = Scheduler(_fake({i: 0.005 for i in range(5)}, log), lambda r: 1, slots=1, budget_bytes=10,
                      policy="smallest")
    sched.serve(reqs, realtime=False)
    starts = [rid for kind, rid, _ in log if kind == "start"]
    assert starts == [1, 4, 2, 0, 3]


def test_smallest_first_skips_what_does_not_fit_and_ages():
    """A large request that does not fit does not block smaller ones; once it
    has waited longer than max_wait it goes first and is not overtaken."""
    big = Request(0, (1, 1, 1), (32, 32, 32), 2, 0, arrival=0.0)
    small = [Request(i, (1, 1, 1), (4, 4, 4), 2, i, arrival=0.0) for i in range(1, 9)]
    log = []
    size = {0: 10}
    size.update({i: 4 for i in range(1, 9)})
    sched = Scheduler(_fake({i: 0.03 for i in range(9)}, log), lambda r: size[r.id], slots=3, budget_bytes=10,
                      policy="smallest", max_wait=0.05)
    sched.serve([big] + small, realtime=True)
    starts = [rid for kind, rid, _ in log if kind == "start"]
    assert starts[0] != 0                       # small ones first while nothing aged
    i_big = starts.index(0)
    assert i_big < len(starts) - 1              # aged: admitted before the small ones are exhausted
    used, peak = 0, 0
    for kind, rid, _ in log:
        used += size[rid] if kind == "start" else -size[rid]
        peak = max(peak, used)
    assert peak <= 10


def test_unknown_policy_is_rejected():
    with pytest.raises(ValueError):
        Scheduler(lambda r, s: {}, lambda r: 1, slots=1, budget_bytes=1, policy="lifo")
