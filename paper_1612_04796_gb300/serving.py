"""Serving: continuous batching of independent Poisson solves.

Requests (periodic box, mesh, order P, right-hand side) arrive over time.
The native runtime (include/mgdg_server.h) admits a request as soon as a
worker slot is free and its device-memory footprint fits into the HBM budget
(first come first served, or smallest work first with aging).  Every
admitted request gets its own solver context, pool memory and CUDA stream on
a worker thread; the solves of different requests therefore overlap on the
GPU, and each result is independent of what else runs (the kernels are
deterministic and share no state), so a request gives the same answer alone
and in the mix.

``Server`` binds the runtime; with an ``executor`` in place of the GPU solve
the same admission code runs without a GPU (tests).
"""
import ctypes
import time

import numpy as np

from . import inputs


POLICY = {"fcfs": 0, "smallest": 1}


class Request:
    def __init__(self, rid, lengths, counts, P, seed, arrival=0.0, tol=1e-10, overlap=1, footprint=0):
        self.id = rid
        self.lengths = tuple(float(v) for v in lengths)
        self.counts = tuple(int(v) for v in counts)
        self.P = int(P)
        self.seed = int(seed)
        self.arrival = float(arrival)
        self.tol = float(tol)
        self.overlap = int(overlap)
        self.footprint = int(footprint)  # bytes; 0 = the library's sizing

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
        self.batch = 1
        self.slot = -1

    @property
    def latency(self):
        return self.t_done - self.t_arrival


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
    """Binding of the native serving runtime (include/mgdg_server.h): the
    admission, the worker threads, the streams and the device memory are the
    library's; this class marshals requests in and results out.

    Real solves by default: FP32 V-cycle preconditioner inside the inexact
    PCG, whose outer iteration runs in double-float arithmetic (outer_df64 =
    "all": vectors, inner products, updates and q = A p in FP32 pairs, the
    convergence confirmed on the FP64 residual; True: only q = A p; False:
    FP64); requests of
    at most ``batch_dofs`` DOFs and the same order are solved in groups of up
    to ``batch_max`` (mg_solve_batch: one launch per sweep for the group).  Each
    request's nodal right-hand side is drawn from its seed when the runtime
    admits it (the fill callback), so queued requests hold no host buffer.

    ``executor(req, slot) -> {"iterations": .., "relres": ..}`` replaces the
    GPU solve (host-only use of the scheduler, e.g. tests); the runtime then
    makes no CUDA call, and ``req.footprint`` (bytes) is the request's size."""

    def __init__(self, slots=8, budget_bytes=None, precision="mixed", use_cg=True, device="cuda", keep_solution=True,
                 outer_df64="all", policy="fcfs", max_wait=10.0, executor=None, maxit=400, batch_max=16,
                 batch_dofs=1 << 20):
        from . import _lib
        from .solver import PRECISION
        if policy not in POLICY:
            raise ValueError("unknown policy %r" % policy)
        self._lib = _lib
        self.lib = _lib.load_library()
        self.precision = precision
        self.outer_df64 = outer_df64 if precision != "fp64" else False
        self.use_cg = use_cg
        self.keep = keep_solution and executor is None
        self.policy = policy
        self.max_wait = float(max_wait)
        self.executor = executor
        o = _lib.MgServerOpts()
        self.lib.mg_server_default_opts(ctypes.byref(o))
        o.slots = int(slots)
        o.policy = POLICY[policy]
        o.max_wait = self.max_wait
        o.use_cg = 1 if use_cg else 0
        o.maxit = int(maxit)
        o.opts.precision = PRECISION[precision]
        o.opts.outer_df64 = {False: 0, True: 1, "all": 2}[self.outer_df64]
        o.budget = 0 if budget_bytes is None else int(budget_bytes)
        o.batch_max = int(batch_max)
        o.batch_dofs = int(batch_dofs)
        self.batch_max, self.batch_dofs = int(batch_max), int(batch_dofs)
        self._records = {}
        self._next_key = 1
        self._errors = {}
        if executor is None:
            import torch
            dev = torch.device(device)
            if dev.index is None:
                dev = torch.device("cuda", torch.cuda.current_device())
            self.device = dev
            o.device = dev.index
            self._execute_cb = None
        else:
            self.device = None
            self._execute_cb = _lib.EXECUTE_FN(self._execute)
            o.execute = self._execute_cb
        self._fill_cb = _lib.FILL_FN(self._fill)
        self.opts = o
        h = ctypes.c_void_p()
        st = self.lib.mg_server_create(ctypes.byref(o), ctypes.byref(h))
        if st != 0:
            raise RuntimeError("mg_server_create failed: %s" % _lib.STATUS_NAMES.get(st, st))
        self.handle = h

    # callbacks, run on the runtime's worker threads
    def _fill(self, user, ticket, ptr, n):
        req = self._records[user][0]
        out = np.ctypeslib.as_array(ptr, shape=(n,))
        inputs.gaussian(n, req.seed, out=out)

    def _execute(self, user, ticket, reqp, slot, itp, relp):
        key = reqp.contents.user
        try:
            out = self.executor(self._records[key][0], slot)
            itp[0] = int(out.get("iterations", 0))
            relp[0] = float(out.get("relres", 0.0))
            return 0
        except Exception as exc:  # recorded on the result, the runtime goes on
            self._errors[key] = repr(exc)
            return 1

    def _request(self, req, key, u):
        q = self._lib.MgRequest()
        q.lx, q.ly, q.lz = req.lengths
        q.nx, q.ny, q.nz = req.counts
        q.P = req.P
        q.overlap = req.overlap
        q.penalty = 2.0
        q.tol = req.tol
        q.f = None
        q.fill = self._fill_cb
        q.user = key
        q.u = u.ctypes.data if u is not None else None
        q.footprint = int(getattr(req, "footprint", 0) or 0)
        return q

    def footprint(self, req):
        """Bytes the runtime reserves for `req` (host only)."""
        out = ctypes.c_size_t()
        st = self.lib.mg_request_footprint(ctypes.byref(self._request(req, 0, None)), ctypes.byref(self.opts.opts),
                                           ctypes.byref(out))
        if st != 0:
            raise ValueError("invalid request %s" % req.id)
        return out.value

    def serve(self, requests, realtime=True):
        """Submit `requests` (at their arrival times, in seconds from now, when
        `realtime`; all at once otherwise) and wait for every result.
        Returns results in request order."""
        keys = []
        for r in requests:
            u = np.empty(r.dofs) if self.keep else None
            keys.append(self._next_key)
            self._records[self._next_key] = (r, u)
            self._next_key += 1
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        tickets = {}
        t0 = time.perf_counter()
        try:
            for i in order:
                r = requests[i]
                if realtime:
                    delay = r.arrival - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                q = self._request(r, keys[i], self._records[keys[i]][1])
                t = ctypes.c_longlong()
                st = self.lib.mg_submit(self.handle, ctypes.byref(q), ctypes.byref(t))
                if st != 0:
                    raise ValueError("request %s rejected (%s): invalid, or larger than the whole budget"
                                     % (r.id, self._lib.STATUS_NAMES.get(st, st)))
                tickets[i] = t.value
        finally:
            results = []
            for i, r in enumerate(requests):
                res = Result(r.id)
                if i in tickets:
                    out = self._lib.MgResult()
                    self.lib.mg_wait(self.handle, tickets[i], -1.0, ctypes.byref(out))
                    res.iterations, res.relres = out.iterations, out.relres
                    res.t_arrival, res.t_admit, res.t_done = out.t_submit, out.t_admit, out.t_done
                    res.concurrency = out.concurrency
                    res.batch = out.batch
                    res.slot = out.slot
                    if out.status != 0:
                        res.error = self._errors.pop(keys[i], None) or "%s: %s" % (
                            self._lib.STATUS_NAMES.get(out.status, out.status), out.error.decode())
                    res.u = self._records[keys[i]][1]
                self._records.pop(keys[i], None)
                results.append(res)
        return results

    def stats(self):
        st = self._lib.MgServerStats()
        self.lib.mg_server_get_stats(self.handle, ctypes.byref(st))
        return st

    @property
    def max_active(self):
        return self.stats().max_running

    @property
    def budget(self):
        return self.stats().budget

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def latency_summary(results):
    lat = np.array([r.latency for r in results if r.error is None])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()), "completed": int(lat.size),
            "failed": int(sum(r.error is not None for r in results))}
