// Serving runtime: independent solves admitted under a slot limit and a
// device-memory budget, each on its own host worker thread, CUDA stream,
// solver context and pool memory.  Host code only; the solves call the
// library's entry points.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mgdg.h"
#include "../../include/mgdg_server.h"

namespace {

constexpr size_t kRounding = size_t(8) << 20;  // pool allocation rounding reserved per request

struct Job {
  long long ticket = 0;
  mg_request req{};
  double work = 0.0;
  size_t footprint = 0;
  bool done = false;
  mg_result res{};
};

}  // namespace

struct mg_server {
  mg_server_opts o{};
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // workers: a submission, a release, shutdown
  std::condition_variable cv_done;  // waiters: a request finished
  std::deque<std::shared_ptr<Job>> waiting;                   // submitted, not admitted, submission order
  std::unordered_map<long long, std::shared_ptr<Job>> jobs;  // uncollected tickets
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  cudaMemPool_t pool = nullptr;
  size_t used = 0, peak = 0;
  int running = 0, max_running = 0;
  long long next_ticket = 1, submitted = 0, completed = 0;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

extern "C" int mg_sched_pick(int policy, double max_wait, double now, size_t budget, size_t used, int n,
                             const double* arrival, const double* work, const size_t* footprint) {
  if (n < 0 || (n > 0 && (!arrival || !work || !footprint))) return -2;
  if (policy != MG_SCHED_FCFS && policy != MG_SCHED_SMALLEST) return -2;
  if (n == 0) return -1;
  auto fits = [&](int i) { return used <= budget && footprint[i] <= budget - used; };
  if (policy == MG_SCHED_FCFS) return fits(0) ? 0 : -1;
  for (int i = 0; i < n; ++i)  // the oldest aged request goes first or nobody does
    if (now - arrival[i] > max_wait) return fits(i) ? i : -1;
  int best = -1;
  for (int i = 0; i < n; ++i)
    if (fits(i) && (best < 0 || work[i] < work[best])) best = i;
  return best;
}

namespace {

// Index in s->waiting of the request to admit, or -1.  Called with s->mu held.
int pick_locked(mg_server* s) {
  const int n = (int)s->waiting.size();
  std::vector<double> arrival(n), work(n);
  std::vector<size_t> fp(n);
  for (int i = 0; i < n; ++i) {
    arrival[i] = s->waiting[i]->res.t_submit;
    work[i] = s->waiting[i]->work;
    fp[i] = s->waiting[i]->footprint;
  }
  return mg_sched_pick(s->o.policy, s->o.max_wait, s->now(), s->budget, s->used, n, arrival.data(), work.data(),
                       fp.data());
}

void set_error(mg_result& r, const char* what, const char* detail) {
  snprintf(r.error, sizeof(r.error), "%s%s%s", what, detail && *detail ? ": " : "", detail ? detail : "");
}

// One request on the GPU: its context, pool memory (workspace, f, b, u) and
// the right-hand side assembled, ready for mg_solve / mg_solve_batch.
struct GpuRun {
  mg_ctx* ctx = nullptr;
  void* bufs[4] = {nullptr, nullptr, nullptr, nullptr};  // workspace, f, b, u
  size_t sizes[4] = {0, 0, 0, 0};
  int status = MG_OK;
  double* b() const { return (double*)bufs[2]; }
  double* u() const { return (double*)bufs[3]; }
};

void gpu_prepare(mg_server* s, Job& job, int slot, GpuRun& g) {
  const mg_request& q = job.req;
  mg_result& r = job.res;
  cudaStream_t st = s->streams[slot];
  mg_opts o = s->o.opts;
  o.stream = (void*)st;
  g.status = mg_setup(q.lx, q.ly, q.lz, q.nx, q.ny, q.nz, q.P, q.penalty, q.overlap, &o, &g.ctx);
  if (g.status != MG_OK) {
    set_error(r, "mg_setup", g.ctx ? mg_last_error(g.ctx) : "");
    return;
  }
  const size_t n = (size_t)mg_num_dofs(g.ctx, mg_num_levels(g.ctx) - 1);
  mg_workspace_size(g.ctx, &g.sizes[0]);
  g.sizes[1] = g.sizes[2] = g.sizes[3] = n * sizeof(double);
  cudaError_t ce = cudaSuccess;
  for (int i = 0; i < 4 && ce == cudaSuccess; ++i) ce = cudaMallocFromPoolAsync(&g.bufs[i], g.sizes[i], s->pool, st);
  if (ce != cudaSuccess) {
    g.status = ce == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA;
    set_error(r, "device allocation", cudaGetErrorString(ce));
    return;
  }
  g.status = mg_bind_workspace(g.ctx, g.bufs[0], g.sizes[0]);
  if (g.status != MG_OK) {
    set_error(r, "mg_bind_workspace", mg_last_error(g.ctx));
    return;
  }
  std::unique_ptr<double[]> fbuf;
  const double* src = q.f;
  if (!src) {
    fbuf.reset(new (std::nothrow) double[n]);
    if (!fbuf) {
      g.status = MG_ENOMEM;
      set_error(r, "host buffer of the right-hand side", "");
      return;
    }
    q.fill(q.user, job.ticket, fbuf.get(), n);
    src = fbuf.get();
  }
  ce = cudaMemcpyAsync(g.bufs[1], src, g.sizes[1], cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(g.u(), 0, g.sizes[3], st);
  if (ce == cudaSuccess && fbuf) ce = cudaStreamSynchronize(st);  // fbuf is released on return
  if (ce != cudaSuccess) {
    g.status = MG_ECUDA;
    set_error(r, "copy in", cudaGetErrorString(ce));
    return;
  }
  g.status = mg_rhs(g.ctx, (const double*)g.bufs[1], g.b());
  if (g.status != MG_OK) set_error(r, "mg_rhs", mg_last_error(g.ctx));
}

// Copy the solution out, release the memory and the context; the request's status.
int gpu_finish(mg_server* s, Job& job, int slot, GpuRun& g) {
  cudaStream_t st = s->streams[slot];
  if ((g.status == MG_OK || g.status == MG_ENOCONV) && job.req.u) {
    const cudaError_t ce = cudaMemcpyAsync(job.req.u, g.u(), g.sizes[3], cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) {
      g.status = MG_ECUDA;
      set_error(job.res, "copy out", cudaGetErrorString(ce));
    }
  }
  for (int i = 0; i < 4; ++i)
    if (g.bufs[i]) cudaFreeAsync(g.bufs[i], st);
  const cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess && g.status == MG_OK) {
    g.status = MG_ECUDA;
    set_error(job.res, "stream", cudaGetErrorString(ce));
  }
  if (g.ctx) mg_destroy(g.ctx);
  return g.status;
}

// The GPU executor: one request with mg_solve, or (batched) a group of one or
// more with mg_solve_batch.
void gpu_solve(mg_server* s, std::vector<std::shared_ptr<Job>>& group, int slot, bool batched) {
  const int n = (int)group.size();
  char label[64];  // NVTX range of the worker's solve (tracing)
  snprintf(label, sizeof(label), "serve slot %d: %d request%s", slot, n, n > 1 ? "s" : "");
  nvtxRangePushA(label);
  std::vector<GpuRun> runs(n);
  for (int i = 0; i < n; ++i) gpu_prepare(s, *group[i], slot, runs[i]);
  std::vector<int> ok;
  for (int i = 0; i < n; ++i)
    if (runs[i].status == MG_OK) ok.push_back(i);
  if (ok.size() == 1 && !batched) {
    Job& j = *group[ok[0]];
    GpuRun& g = runs[ok[0]];
    g.status = mg_solve(g.ctx, g.u(), g.b(), j.req.tol, s->o.maxit, s->o.use_cg, &j.res.iterations, &j.res.relres,
                        nullptr);
    if (g.status != MG_OK) set_error(j.res, "mg_solve", mg_last_error(g.ctx));
  } else if (!ok.empty()) {
    const int k = (int)ok.size();
    std::vector<mg_ctx*> ctxs(k);
    std::vector<double*> us(k);
    std::vector<const double*> bs(k);
    std::vector<int> its(k), sts(k);
    std::vector<double> rel(k);
    for (int i = 0; i < k; ++i) {
      ctxs[i] = runs[ok[i]].ctx;
      us[i] = runs[ok[i]].u();
      bs[i] = runs[ok[i]].b();
    }
    const int st = mg_solve_batch(ctxs.data(), k, us.data(), bs.data(), group[ok[0]]->req.tol, s->o.maxit,
                                  its.data(), rel.data(), sts.data());
    for (int i = 0; i < k; ++i) {
      Job& j = *group[ok[i]];
      GpuRun& g = runs[ok[i]];
      j.res.iterations = its[i];
      j.res.relres = rel[i];
      g.status = st != MG_OK ? st : sts[i];
      if (g.status != MG_OK) set_error(j.res, "mg_solve_batch", st != MG_OK ? mg_last_error(ctxs[0]) : "");
    }
  }
  for (int i = 0; i < n; ++i) group[i]->res.status = gpu_finish(s, *group[i], slot, runs[i]);
  nvtxRangePop();
}

void worker(mg_server* s, int slot) {
  if (!s->o.execute) cudaSetDevice(s->o.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    std::shared_ptr<Job> job;
    for (;;) {
      if (!s->waiting.empty()) {
        const int k = pick_locked(s);
        if (k >= 0) {
          job = s->waiting[k];
          s->waiting.erase(s->waiting.begin() + k);
          break;
        }
      } else if (s->stop) {
        return;
      }
      s->cv_work.wait(lk);
    }
    // batching: small requests take the batched path, with further waiting
    // requests of the same order and tolerance, all small
    std::vector<std::shared_ptr<Job>> group{job};
    const bool batched = !s->o.execute && s->o.use_cg && job->work <= (double)s->o.batch_dofs;
    if (batched && s->o.batch_max > 1) {
      size_t held = s->used + job->footprint;
      for (auto it = s->waiting.begin(); it != s->waiting.end() && (int)group.size() < s->o.batch_max;) {
        const Job& c = **it;
        if (c.req.P == job->req.P && c.req.tol == job->req.tol && c.work <= (double)s->o.batch_dofs &&
            c.footprint <= s->budget - held) {
          held += c.footprint;
          group.push_back(*it);
          it = s->waiting.erase(it);
        } else {
          ++it;
        }
      }
    }
    const double t_admit = s->now();
    for (auto& j : group) {
      s->used += j->footprint;
      s->running += 1;
      j->res.t_admit = t_admit;
      j->res.slot = slot;
      j->res.batch = (int)group.size();
    }
    s->peak = std::max(s->peak, s->used);
    s->max_running = std::max(s->max_running, s->running);
    for (auto& j : group) j->res.concurrency = s->running;
    lk.unlock();

    if (s->o.execute) {
      const int status = s->o.execute(s->o.execute_user, job->ticket, &job->req, slot, &job->res.iterations,
                                      &job->res.relres);
      if (status != MG_OK && !job->res.error[0]) set_error(job->res, "executor", "");
      job->res.status = status;
    } else {
      gpu_solve(s, group, slot, batched);
    }

    lk.lock();
    const double t_done = s->now();
    for (auto& j : group) {
      j->res.t_done = t_done;
      j->done = true;
      s->used -= j->footprint;
      s->running -= 1;
      s->completed += 1;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
}

bool valid_opts(const mg_server_opts* o) {
  return o->slots >= 1 && o->slots <= 256 && (o->policy == MG_SCHED_FCFS || o->policy == MG_SCHED_SMALLEST) &&
         o->max_wait >= 0.0 && o->maxit >= 1 && (o->use_cg == 0 || o->use_cg == 1) && o->device >= 0 &&
         o->batch_max >= 1 && o->batch_max <= 16;
}

// The library's sizing of a request (host only), or 0 if mg_setup rejects it.
size_t library_footprint(const mg_request* q, const mg_opts* opts, int* status) {
  mg_ctx* ctx = nullptr;
  *status = mg_setup(q->lx, q->ly, q->lz, q->nx, q->ny, q->nz, q->P, q->penalty, q->overlap, opts, &ctx);
  if (*status != MG_OK) {
    if (ctx) mg_destroy(ctx);
    return 0;
  }
  size_t ws = 0;
  mg_workspace_size(ctx, &ws);
  const size_t n = (size_t)mg_num_dofs(ctx, mg_num_levels(ctx) - 1);
  mg_destroy(ctx);
  return ws + 3 * n * sizeof(double) + kRounding;
}

}  // namespace

extern "C" {

void mg_server_default_opts(mg_server_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->slots = 8;
  o->budget = 0;
  o->policy = MG_SCHED_FCFS;
  o->max_wait = 10.0;
  o->device = 0;
  o->use_cg = 1;
  o->maxit = 400;
  mg_default_opts(&o->opts);
  o->batch_max = 16;
  o->batch_dofs = size_t(1) << 20;
}

mg_status mg_request_footprint(const mg_request* req, const mg_opts* opts, size_t* bytes) {
  if (!req || !bytes) return MG_EINVAL;
  mg_opts d;
  if (!opts) {
    mg_default_opts(&d);
    opts = &d;
  }
  int st = MG_OK;
  const size_t fp = library_footprint(req, opts, &st);
  if (st != MG_OK) return (mg_status)st;
  *bytes = std::max(fp, req->footprint);
  return MG_OK;
}

mg_status mg_server_create(const mg_server_opts* opts, mg_server** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  mg_server_opts o;
  if (opts) o = *opts;
  else mg_server_default_opts(&o);
  if (!valid_opts(&o)) return MG_EINVAL;
  std::unique_ptr<mg_server> s(new (std::nothrow) mg_server());
  if (!s) return MG_ENOMEM;
  s->o = o;
  s->o.opts.stream = nullptr;
  s->budget = o.budget;
  if (!o.execute) {
    if (cudaSetDevice(o.device) != cudaSuccess) return MG_ECUDA;
    if (s->budget == 0) {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return MG_ECUDA;
      s->budget = (size_t)(0.8 * (double)free_b);
    }
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = o.device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) return MG_ECUDA;
    uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool for the next request
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    s->streams.resize(o.slots, nullptr);
    for (int i = 0; i < o.slots; ++i) {
      if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaStreamDestroy(s->streams[j]);
        cudaMemPoolDestroy(s->pool);
        return MG_ECUDA;
      }
    }
  } else if (s->budget == 0) {
    s->budget = SIZE_MAX;
  }
  s->t0 = std::chrono::steady_clock::now();
  mg_server* raw = s.release();
  for (int i = 0; i < o.slots; ++i) raw->workers.emplace_back(worker, raw, i);
  *out = raw;
  return MG_OK;
}

mg_status mg_submit(mg_server* s, const mg_request* req, long long* ticket) {
  if (!s || !req || !ticket) return MG_EINVAL;
  if (!req->f && !req->fill) return MG_EINVAL;
  if (!(req->tol > 0.0)) return MG_EINVAL;
  int st = MG_OK;
  const size_t lib_fp = library_footprint(req, &s->o.opts, &st);
  if (st != MG_OK) return (mg_status)st;
  auto job = std::make_shared<Job>();
  job->req = *req;
  job->footprint = s->o.execute ? (req->footprint ? req->footprint : lib_fp) : std::max(lib_fp, req->footprint);
  if (job->footprint > s->budget) return MG_EINVAL;
  job->work = (double)req->nx * req->ny * req->nz * (double)(req->P + 1) * (req->P + 1) * (req->P + 1);
  job->res.footprint = job->footprint;
  job->res.slot = -1;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return MG_EINVAL;
  job->ticket = s->next_ticket++;
  job->res.t_submit = s->now();
  s->waiting.push_back(job);
  s->jobs[job->ticket] = job;
  s->submitted += 1;
  *ticket = job->ticket;
  s->cv_work.notify_all();
  return MG_OK;
}

static mg_status collect_locked(mg_server* s, long long ticket, mg_result* out, bool* found) {
  auto it = s->jobs.find(ticket);
  *found = it != s->jobs.end();
  if (!*found) return MG_EINVAL;
  if (!it->second->done) return MG_ENOTREADY;
  *out = it->second->res;
  s->jobs.erase(it);
  return MG_OK;
}

mg_status mg_poll(mg_server* s, long long ticket, mg_result* out) {
  if (!s || !out) return MG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  bool found;
  return collect_locked(s, ticket, out, &found);
}

mg_status mg_wait(mg_server* s, long long ticket, double timeout_s, mg_result* out) {
  if (!s || !out) return MG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return MG_EINVAL;
  std::shared_ptr<Job> job = it->second;
  if (timeout_s < 0) {
    s->cv_done.wait(lk, [&] { return job->done; });
  } else {
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return job->done; });
  }
  bool found;
  return collect_locked(s, ticket, out, &found);
}

mg_status mg_server_get_stats(mg_server* s, mg_server_stats* out) {
  if (!s || !out) return MG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->queued = (int)s->waiting.size();
  out->running = s->running;
  out->max_running = s->max_running;
  out->budget = s->budget;
  out->used = s->used;
  out->peak_used = s->peak;
  return MG_OK;
}

void mg_server_destroy(mg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  for (auto& t : s->workers) t.join();
  if (!s->o.execute) {
    cudaSetDevice(s->o.device);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (s->pool) cudaMemPoolDestroy(s->pool);
  }
  delete s;
}

}  // extern "C"
