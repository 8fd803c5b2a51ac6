/*
 * mgdg_server.h -- C ABI of the serving runtime: a queue of independent
 * periodic Poisson solves (each one the problem of mgdg.h: box, mesh, order P,
 * nodal right-hand side) run concurrently on one GPU.
 *
 * The paper solves one problem at a time; this runtime is the library's own
 * addition.  Each admitted request gets its own solver context, device
 * memory and CUDA stream on one of `slots` host worker threads, so the solves
 * of different requests overlap on the GPU.  The kernels are deterministic
 * and share no state, so a request's result does not depend on what else
 * runs.
 *
 * Admission (mg_sched_pick): a request is admitted when a worker is free and
 * its device-memory footprint fits into what the budget has left.
 *   MG_SCHED_FCFS      strictly in submission order; a request that does not
 *                      fit blocks the ones behind it (large ones never starve).
 *   MG_SCHED_SMALLEST  the waiting request with the least work (DOFs) that
 *                      fits goes first (ties: earliest); a request that has
 *                      waited longer than max_wait seconds is aged: the aged
 *                      ones go first, in submission order, and are not
 *                      overtaken even when they do not fit yet.
 *
 * Memory: the server owns the device memory of its requests.  It comes from
 * a stream-ordered pool of the server's own (cudaMemPoolCreate; freed memory
 * stays in the pool for the next request) and is released by
 * mg_server_destroy.  The footprint of a request is the library's workspace
 * size (mg_workspace_size) plus three FP64 vectors of N DOFs (nodal f, weak
 * rhs b, solution u) plus 8 MiB of allocation rounding.
 *
 * Threads: every function may be called from any host thread.  A request's
 * host buffers (f, u) must stay valid until its result has been collected.
 * Errors are status codes (mg_status of mgdg.h); a failed solve is reported in
 * its result and does not stop the server.
 */
#ifndef MGDG_SERVER_H
#define MGDG_SERVER_H

#include <stddef.h>

#include "mgdg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_server mg_server;

typedef enum { MG_SCHED_FCFS = 0, MG_SCHED_SMALLEST = 1 } mg_sched_policy;

/* One solve: the arguments of mg_setup, the tolerance of mg_solve and the
 * nodal right-hand side on the host. */
typedef struct {
  double lx, ly, lz;  /* box lengths (> 0) */
  int nx, ny, nz;     /* elements per direction */
  int P;              /* polynomial order */
  int overlap;        /* N_O node layers of the smoother (mg_setup) */
  double penalty;     /* mu / mu_min (mg_setup; the paper's choice is 2) */
  double tol;         /* relative residual reduction (mg_solve) */
  /* Nodal right-hand side f (N = nx ny nz (P+1)^3 doubles, element-blocked),
   * given one of two ways: `f` points to it (host memory, caller-owned until
   * the result is collected), or `f` is NULL and `fill` is called on the worker
   * thread when the request is admitted to write it into a host buffer of the
   * server's (so queued requests hold no right-hand side).  `user` is passed
   * to `fill` unchanged. */
  const double* f;
  void (*fill)(void* user, long long ticket, double* f, size_t n);
  void* user;
  double* u;          /* host, N doubles: receives the solution; NULL = not copied back */
  size_t footprint;   /* 0, or bytes the request holds while it runs: with the GPU
                         executor the larger of this and the library's sizing is used;
                         with a custom executor this value as given */
} mg_request;

typedef struct {
  int slots;          /* concurrent solves: host worker threads, one CUDA stream each (1 .. 256) */
  size_t budget;      /* device bytes the running requests may hold together;
                         0 = 80 % of the free device memory at mg_server_create */
  int policy;         /* mg_sched_policy */
  double max_wait;    /* seconds before a request is aged (MG_SCHED_SMALLEST) */
  int device;         /* CUDA device ordinal */
  int use_cg;         /* mg_solve: 1 MG-CG (default), 0 standalone V-cycles */
  int maxit;          /* mg_solve iteration limit (default 400) */
  mg_opts opts;       /* solver options of every request (precision, overlap mode, ...);
                         opts.stream is ignored: each worker has its own stream */
  /* Executor: NULL = the GPU solve (setup, workspace, H2D copy of f, mg_rhs,
   * mg_solve from u = 0, D2H copy of u).  Otherwise called on the worker thread
   * instead, with the worker's slot; it returns an mg_status and may set
   * *iterations and *relres.  With a custom executor the server makes no CUDA
   * call at all (budget 0 then means unlimited). */
  int (*execute)(void* user, long long ticket, const mg_request* req, int slot, int* iterations,
                 double* relres);
  void* execute_user;
  /* Batching (GPU executor, use_cg = 1): requests of at most batch_dofs DOFs
   * are solved with mg_solve_batch (every sweep one launch for the group); a
   * worker that admits one also admits, in submission order, further waiting
   * requests of the same order P and tolerance, of at most batch_dofs DOFs,
   * that fit into the budget, up to batch_max in all.  A small request's
   * result is therefore the same bits whatever it was grouped with (and equal
   * to a separate mg_solve to rounding).  batch_max 1 = groups of one
   * (1 .. 16); batch_dofs 0 = no request takes the batched path. */
  int batch_max;
  size_t batch_dofs;
} mg_server_opts;

typedef struct {
  int status;         /* mg_status of the solve */
  int iterations;     /* mg_solve's iteration count */
  double relres;      /* final relative residual */
  double t_submit, t_admit, t_done;  /* seconds since mg_server_create (monotonic clock) */
  int concurrency;    /* requests running when this one was admitted, itself included */
  int batch;          /* requests solved together with it (mg_solve_batch), itself included */
  int slot;           /* worker that ran it */
  size_t footprint;   /* bytes it held */
  char error[160];    /* message of a failed solve, else empty */
} mg_result;

typedef struct {
  long long submitted, completed;
  int queued, running, max_running;
  size_t budget, used, peak_used;
} mg_server_stats;

/* Defaults: 8 slots, budget 0, MG_SCHED_FCFS, max_wait 10 s, device 0, use_cg 1,
 * maxit 400, mg_default_opts, GPU executor, batch_max 16, batch_dofs 2^20. */
void mg_server_default_opts(mg_server_opts* o);

/* Start the workers.  MG_EINVAL for a bad option, MG_ECUDA if the device,
 * streams or pool cannot be set up. */
mg_status mg_server_create(const mg_server_opts* opts, mg_server** out);

/* Footprint (bytes) the GPU executor reserves for `req` under solver options
 * `opts` (NULL = defaults): host only, no CUDA call.  MG_EINVAL for a request
 * that mg_setup rejects. */
mg_status mg_request_footprint(const mg_request* req, const mg_opts* opts, size_t* bytes);

/* Queue a request (the descriptor is copied).  *ticket identifies it.
 * MG_EINVAL for an invalid request (mg_setup's checks, no f and no fill), one
 * whose footprint exceeds the whole budget, or a server being destroyed. */
mg_status mg_submit(mg_server* s, const mg_request* req, long long* ticket);

/* Result of a finished request: MG_OK and *out filled (the ticket is then
 * released: a second call gives MG_EINVAL); MG_ENOTREADY while it is queued
 * or running; MG_EINVAL for an unknown ticket. */
mg_status mg_poll(mg_server* s, long long ticket, mg_result* out);

/* Like mg_poll, but waits up to timeout_s seconds (< 0: no limit) for the
 * request to finish; MG_ENOTREADY if it has not by then. */
mg_status mg_wait(mg_server* s, long long ticket, double timeout_s, mg_result* out);

/* Counters since creation. */
mg_status mg_server_get_stats(mg_server* s, mg_server_stats* out);

/* Finish every submitted request, stop the workers and release the streams
 * and the pool.  Uncollected results are discarded. */
void mg_server_destroy(mg_server* s);

/*
 * mg_sched_pick -- the admission rule (host only): index of the request to
 * admit next among n waiting ones (in submission order: arrival[i] seconds,
 * work[i], footprint[i] bytes), at time `now`, with `used` of `budget` bytes
 * held; -1 if none may be admitted now; -2 for bad arguments.
 */
int mg_sched_pick(int policy, double max_wait, double now, size_t budget, size_t used, int n,
                  const double* arrival, const double* work, const size_t* footprint);

#ifdef __cplusplus
}
#endif

#endif /* MGDG_SERVER_H */
