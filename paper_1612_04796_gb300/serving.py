"""Serving loop: continuous batching of independent Poisson solves.

Requests (periodic box, mesh, order P, right-hand side) arrive over time.  A
request is admitted as soon as a worker slot is free and its device-memory
footprint fits into the HBM budget (first come, first served: a request that
does not fit blocks the ones behind it, so large requests are not starved).
Every admitted request gets its own solver context, workspace and CUDA
stream on a worker thread; the solves of different requests therefore
overlap on the GPU, and each result is independent of what else runs (the
kernels are deterministic and share no state), so a request gives the same
answer alone and in the mix.

The scheduling logic (``Scheduler``) is separate from the GPU work so that it
can be tested with fake solves; ``Server`` plugs in the real solver.
"""
import collections
import ctypes
import threading
import time

import numpy as np

from . import inputs


class Request:
    def __init__(self, rid, lengths, counts, P, seed, arrival=0.0, tol=1e-10, overlap=1):
        self.id = rid
        self.lengths = tuple(float(v) for v in lengths)
        self.counts = tuple(int(v) for v in counts)
        self.P = int(P)
        self.seed = int(seed)
        self.arrival = float(arrival)
        self.tol = float(tol)
        self.overlap = int(overlap)

    @property
    def dofs(self):
        return self.counts[0] * self.counts[1] * self.counts[2] * (self.P + 1) ** 3


class Result:
    def __init__(self, rid):
        self.id = rid
        self.u = None
        self.iterations = None
        self.relres = None
        self.t_arrival = None
        self.t_admit = None
        self.t_done = None
        self.error = None
        self.concurrency = 0

    @property
    def latency(self):
        return self.t_done - self.t_arrival


class Scheduler:
    """Admission under a slot limit and a memory budget.  ``footprint(req)``
    gives the bytes a request holds while it runs; ``run(req, slot)`` does the
    work (on a worker thread) and returns a dict that is stored on the Result.

    policy "fcfs": strictly in arrival order (a request that does not fit
    blocks the ones behind it).  policy "smallest": among the requests that
    have arrived, the one with the least work (``work(req)``, default its DOF
    count) that fits is admitted first; a request that has waited longer than
    ``max_wait`` seconds is aged: the aged ones go first, in arrival order and
    without being overtaken, so no request waits much longer than max_wait
    for its turn."""

    def __init__(self, run, footprint, slots, budget_bytes, clock=time.perf_counter, policy="fcfs", work=None,
                 max_wait=10.0):
        if policy not in ("fcfs", "smallest"):
            raise ValueError("unknown policy %r" % policy)
        self.run = run
        self.footprint = footprint
        self.slots = int(slots)
        self.budget = int(budget_bytes)
        self.clock = clock
        self.policy = policy
        self.work = work if work is not None else (lambda r: r.dofs)
        self.max_wait = float(max_wait)
        self.cv = threading.Condition()
        self.used = 0
        self.active = 0
        self.max_active = 0
        self.free_slots = list(range(self.slots))

    def _worker(self, req, slot, res, need):
        try:
            out = self.run(req, slot)
            for k, v in out.items():
                setattr(res, k, v)
        except Exception as exc:  # recorded on the result, the loop goes on
            res.error = repr(exc)
        res.t_done = self.clock()
        with self.cv:
            self.used -= need
            self.active -= 1
            self.free_slots.append(slot)
            self.cv.notify_all()

    def _pick(self, waiting, now, realtime):
        """The request to admit next among `waiting` (arrived, not admitted),
        or None to wait for resources.  Called with self.cv held."""
        fits = lambda r: self.used + self.footprint(r) <= self.budget
        if self.policy == "fcfs":
            return waiting[0] if fits(waiting[0]) else None
        aged = [r for r in waiting if realtime and now - r.arrival > self.max_wait]
        if aged:
            return aged[0] if fits(aged[0]) else None
        best = None
        for r in waiting:
            if fits(r) and (best is None or self.work(r) < self.work(best)):
                best = r
        return best

    def serve(self, requests, realtime=True):
        """Serve `requests` (arrival in seconds from the start).  Returns
        results in request order."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = []
        results = {r.id: Result(r.id) for r in requests}
        t0 = self.clock()
        threads = []
        for r in requests:
            if self.footprint(r) > self.budget:
                raise ValueError("request %s needs more memory than the whole budget" % r.id)
        while pending or waiting:
            now = self.clock() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.popleft())
            if not waiting:
                time.sleep(min(pending[0].arrival - now, 0.005))
                continue
            with self.cv:
                req = self._pick(waiting, self.clock() - t0, realtime) if self.free_slots else None
                if req is None:
                    self.cv.wait(timeout=0.005 if pending else 0.05)
                    continue
                need = self.footprint(req)
                slot = self.free_slots.pop(0)
                self.used += need
                self.active += 1
                self.max_active = max(self.max_active, self.active)
                active_now = self.active
            waiting.remove(req)
            res = results[req.id]
            res.t_arrival = t0 + (req.arrival if realtime else 0.0)
            res.t_admit = self.clock()
            res.concurrency = active_now
            th = threading.Thread(target=self._worker, args=(req, slot, res, need), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        return [results[r.id] for r in requests]


def request_stream(seed=5, n_requests=512, rate=200.0, sizes=(4, 8, 16, 24, 32), orders=(2, 4, 8, 16),
                   aspect=(1.0, 8.0), overlap=1):
    """The serving workload: Poisson arrivals, box [0, AR] x [0, 1] x [0, 1]
    with n^3 elements, order P, Gaussian right-hand side from a per-request
    seed; `overlap` = N_O node layers of every request's smoother."""
    reqs = []
    for i, d in enumerate(inputs.request_stream(seed, n_requests, rate, sizes, orders, aspect)):
        reqs.append(Request(i, (d["aspect"], 1.0, 1.0), (d["n"],) * 3, d["P"], d["seed"], d["arrival"],
                            overlap=overlap))
    return reqs


class Server:
    """Real solves: FP32 V-cycle preconditioner inside FP64 inexact PCG by
    default, the outer products q = A p in double-float (outer_df64); each
    slot owns a CUDA stream."""

    def __init__(self, slots=8, budget_bytes=None, precision="mixed", use_cg=True, device="cuda", keep_solution=True,
                 outer_df64=True, policy="fcfs", max_wait=10.0):
        import torch

        from ._lib import MgOpts, load_library
        from .solver import MGSolver
        self.torch = torch
        self.MGSolver = MGSolver
        self.lib = load_library()
        self.MgOpts = MgOpts
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.8 * free)
        self.precision = precision
        self.outer_df64 = bool(outer_df64) and precision != "fp64"
        self.use_cg = use_cg
        self.keep = keep_solution
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.scheduler = Scheduler(self._run, self.footprint, slots, budget_bytes, policy=policy, max_wait=max_wait)

    def footprint(self, req):
        """Workspace plus the request's own vectors (f, b, u), from the
        library's host-only sizing."""
        opts = self.MgOpts()
        self.lib.mg_default_opts(ctypes.byref(opts))
        ctx = ctypes.c_void_p()
        st = self.lib.mg_setup(req.lengths[0], req.lengths[1], req.lengths[2], req.counts[0], req.counts[1],
                               req.counts[2], req.P, 2.0, req.overlap, ctypes.byref(opts), ctypes.byref(ctx))
        if st != 0:
            raise ValueError("invalid request %s" % req.id)
        size = ctypes.c_size_t()
        self.lib.mg_workspace_size(ctx, ctypes.byref(size))
        self.lib.mg_destroy(ctx)
        return size.value + 3 * 8 * req.dofs + (1 << 20)

    def _run(self, req, slot):
        torch = self.torch
        stream = self.streams[slot]
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            s = self.MGSolver(req.lengths, req.counts, req.P, overlap=req.overlap, precision=self.precision,
                              device=self.device, stream=stream, outer_df64=self.outer_df64)
            f = torch.tensor(inputs.gaussian(s.num_dofs(), req.seed), device=self.device)
            b = s.rhs(f)
            u, its, rel, _ = s.solve(b, tol=req.tol, use_cg=self.use_cg, maxit=400)
            out = u.cpu().numpy() if self.keep else None
            stream.synchronize()
            s.close()
            del s, f, b, u
        return {"u": out, "iterations": its, "relres": rel}

    def serve(self, requests, realtime=True):
        return self.scheduler.serve(requests, realtime)

    @property
    def max_active(self):
        return self.scheduler.max_active


def latency_summary(results):
    lat = np.array([r.latency for r in results if r.error is None])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()), "completed": int(lat.size),
            "failed": int(sum(r.error is not None for r in results))}
