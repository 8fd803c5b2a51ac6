// C ABI entry points and host orchestration of the multigrid solver.
//
// mg_setup derives the level hierarchy P_l = 2^l (Section 3.2), the overlap of
// every level (Section 3.1, Table 1) and the workspace layout; the device
// builds all tables at mg_bind_workspace.  mg_vcycle follows Algorithm 1,
// mg_solve repeats it (MG) or uses it as the preconditioner of the inexact
// preconditioned CG (MG-CG, Section 3.2); residual norms are Euclidean
// (Section 4).
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mg_internal.h"

using namespace mgdg;

namespace {

mg_status fail(mg_ctx* c, mg_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

mg_status cuda_fail(mg_ctx* c, cudaError_t e, const char* what) {
  return fail(c, MG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);  \
  } while (0)

// ---- host-side GLL nodes, used only to size the hierarchy (overlap layers) ----
double legendre_host(int P, double x, double* dl) {
  double l0 = 1.0, l1 = x;
  for (int k = 1; k < P; ++k) {
    double l2 = ((2.0 * k + 1.0) * x * l1 - k * l0) / (k + 1.0);
    l0 = l1;
    l1 = l2;
  }
  *dl = P * (x * l1 - l0) / (x * x - 1.0);
  return l1;
}

std::vector<double> gll_host(int P) {
  const double pi = 3.14159265358979323846;
  std::vector<double> x(P + 1);
  x[0] = -1.0;
  x[P] = 1.0;
  for (int k = 1; k < P; ++k) {
    double t = -cos(pi * k / P);
    for (int it = 0; it < 100; ++it) {
      double dl;
      double lp = legendre_host(P, t, &dl);
      double d2 = (2.0 * t * dl - P * (P + 1.0) * lp) / (1.0 - t * t);
      double dt = dl / d2;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[k] = t;
  }
  for (int k = 0; k <= P / 2; ++k) {
    double s = 0.5 * (x[P - k] - x[k]);
    x[k] = -s;
    x[P - k] = s;
  }
  if (P % 2 == 0) x[P / 2] = 0.0;
  return x;
}

// N_O of a geometric overlap delta_O = frac * dx: neighbour nodes with
// distance 1 + xi_k <= 2 frac from the interface (inclusive; Table 1).
int layers_from_width(int P, double frac) {
  std::vector<double> x = gll_host(P);
  int cnt = 0;
  for (double v : x)
    if (1.0 + v <= 2.0 * frac + 1e-12) ++cnt;
  return cnt;
}

// Hat-weight half-width for a strip of N_O neighbour node layers (reference
// units, capped at 1): MG_DELTA_MID, midway between the last included and the
// first excluded neighbour node; MG_DELTA_NODE, the distance of the last
// included node (its weight becomes 0).
double layer_delta(int P, int no, int rule) {
  if (no <= 0) return 0.0;
  std::vector<double> x = gll_host(P);
  if (no >= P + 1) return 1.0;
  double d = rule == MG_DELTA_NODE ? 1.0 + x[no - 1] : 0.5 * ((1.0 + x[no - 1]) + (1.0 + x[no]));
  return d < 1.0 ? d : 1.0;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---- workspace layout ----
struct Layout {
  size_t tab64, tab32, tabdf, lev_u[kMaxLevels], lev_f[kMaxLevels], lev_r[kMaxLevels], corr, ca, cb, cf, cu, cg[8], red,
      scal, status, jac, gjac, total;
  int64_t jac_count, gjac_line, gjac_coarse;
};

Layout make_layout(const mg_ctx* c) {
  Layout ly;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  ly.tab64 = take(c->ws.tab_count * sizeof(double));
  ly.tab32 = take(c->ws.tab_count * sizeof(float));
  ly.tabdf = take(c->ws.tab_count * sizeof(df64));
  int64_t corr = 0;
  for (int l = 0; l <= c->L; ++l) {
    const LevelInfo& lv = c->lev[l];
    ly.lev_u[l] = take(lv.N * sizeof(double));
    ly.lev_f[l] = take(lv.N * sizeof(double));
    ly.lev_r[l] = take(lv.N * sizeof(double));
    if (l >= 1) corr = std::max<int64_t>(corr, c->Ne * (int64_t)lv.m[0] * lv.m[1] * lv.m[2]);
  }
  corr = std::max<int64_t>(corr, 2 * c->lev[c->L].N);
  ly.corr = take(corr * sizeof(double));
  const int64_t N0 = c->lev[0].N, NL = c->lev[c->L].N;
  ly.ca = take(N0 * sizeof(double));
  ly.cb = take(N0 * sizeof(double));
  ly.cf = take(N0 * sizeof(double));
  ly.cu = take(N0 * sizeof(double));
  for (int k = 0; k < 8; ++k) ly.cg[k] = take(NL * sizeof(double));
  ly.red = take(8 * kRedBlocks * sizeof(double));  // up to 5 partial-sum columns
  ly.scal = take(kNumSlots * sizeof(double));
  ly.status = take(256);
  int nmax = 8;
  for (int l = 1; l <= c->L; ++l)
    for (int d = 0; d < 3; ++d) nmax = std::max(nmax, c->lev[l].m[d]);
  for (int d = 0; d < 3; ++d) nmax = std::max(nmax, c->Ng[d]);
  int64_t per_block = 4 * (int64_t)nmax * nmax + 4 * nmax + 64;
  ly.jac_count = per_block * 3 * (c->L + 1);
  ly.jac = take(ly.jac_count * sizeof(double));
  ly.gjac = 0;
  ly.gjac_line = ly.gjac_coarse = 0;
  if (c->graded) {
    // one block per element line of every level (C, V: m^2 each, M: m) and
    // one per coarse direction (Ng^2, Ng^2, Ng)
    int mmax = 1, ngmax = 1;
    for (int l = 1; l <= c->L; ++l)
      for (int d = 0; d < 3; ++d) mmax = std::max(mmax, c->lev[l].m[d]);
    for (int d = 0; d < 3; ++d) ngmax = std::max(ngmax, c->Ng[d]);
    ly.gjac_line = 2 * (int64_t)mmax * mmax + mmax + 32;
    ly.gjac_coarse = 2 * (int64_t)ngmax * ngmax + ngmax + 32;
    const int64_t lines = (int64_t)(c->L + 1) * (c->ne[0] + c->ne[1] + c->ne[2]);
    ly.gjac = take((lines * ly.gjac_line + 3 * ly.gjac_coarse) * sizeof(double));
  }
  ly.total = off;
  return ly;
}

bool check_level(mg_ctx* c, int level, bool need_smoother) {
  if (level < 0 || level > c->L) {
    fail(c, MG_EINVAL, "level out of range");
    return false;
  }
  if (need_smoother && level < 1) {
    fail(c, MG_EINVAL, "level 0 has no smoother / transfer");
    return false;
  }
  return true;
}

mg_status need_ready(mg_ctx* c) {
  if (!c) return MG_EINVAL;
  if (!c->ready) return fail(c, MG_ENOTREADY, "workspace not bound");
  return MG_OK;
}

double read_scalar(mg_ctx* c, int slot, cudaError_t* err) {
  double v = 0.0;
  *err = cudaMemcpyAsync(&v, c->ws.scal + slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (*err == cudaSuccess) *err = cudaStreamSynchronize(c->stream);
  return v;
}

// CUDA events around one kernel group when profiling is on (mg_profile).
// NVTX ranges (tracing): whole solves and every kernel group of the cycle
// appear by name in a profiler's timeline; without a tool attached the calls
// return at once.
const char* const kRangeNames[kProfKinds] = {"smoother FDM", "smoother scatter", "operator", "restriction",
                                             "prolongation", "coarse solve", "vector pass", "outer operator"};

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct ProfScope {
  const mg_ctx* c;
  long idx = -1;
  NvtxRange range;
  ProfScope(const mg_ctx* c_, int kind, int level) : c(c_), range(kRangeNames[kind]) {
    if (!c->prof_on) return;
    if (c->prof_used == c->prof.size()) {
      mg_ctx::ProfRec r{kind, level, nullptr, nullptr};
      if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
      c->prof.push_back(r);
    }
    idx = (long)c->prof_used++;
    c->prof[idx].kind = kind;
    c->prof[idx].level = level;
    cudaEventRecord(c->prof[idx].a, c->stream);
  }
  ~ProfScope() {
    if (idx >= 0) cudaEventRecord(c->prof[idx].b, c->stream);
  }
};

// Run `body` (stream-ordered launches on c->stream, no host synchronisation)
// through a cached CUDA graph: captured once on an internal stream, replayed
// on the caller's stream.  Eager when graphs are off or profiling is on.
template <typename F>
cudaError_t run_graph(mg_ctx* c, int kind, const void* a, const void* b, F body) {
  if (!c->use_graphs || c->prof_on) return body();
  for (auto& g : c->graphs) {
    if (g.kind == kind && g.a == a && g.b == b) {
      c->nlaunch += g.kernels;
      return cudaGraphLaunch(g.exec, c->stream);
    }
  }
  cudaError_t e;
  if (!c->cap_stream && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return e;
  cudaStream_t user = c->stream;
  const long long n0 = c->nlaunch;
  c->stream = c->cap_stream;
  if ((e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
    c->stream = user;
    return e;
  }
  cudaError_t eb = body();
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
  c->stream = user;
  const long long kernels = c->nlaunch - n0;
  c->nlaunch = n0;
  if (eb != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return eb != cudaSuccess ? eb : ee;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  if (c->graphs.size() >= 16) {
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back({kind, a, b, exec, kernels});
  c->nlaunch += kernels;
  return cudaGraphLaunch(exec, c->stream);
}

enum GraphKind : int { kGraphMgCycle = 1, kGraphPrecond, kGraphVcycle, kGraphVcycle32, kGraphCgA, kGraphCgB,
                       kGraphOdfA, kGraphOdfB };

// ---- level vector views ----
template <typename T>
T* lvec(void* p) {
  return static_cast<T*>(p);
}

template <typename T>
cudaError_t coarse_solve_t(const mg_ctx* c, const T* f0, T* u0);
template <>
cudaError_t coarse_solve_t<double>(const mg_ctx* c, const double* f0, double* u0) {
  return launch_coarse_solve(c, f0, u0);
}
template <>
cudaError_t coarse_solve_t<float>(const mg_ctx* c, const float* f0, float* u0) {
  return launch_coarse_solve_f32(c, f0, u0);
}
template <>
cudaError_t coarse_solve_t<df64>(const mg_ctx* c, const df64* f0, df64* u0) {
  return launch_coarse_solve_df64(c, f0, u0);
}

int steps_on_level(const mg_ctx* c, int ns, int l) {
  int s = ns;
  for (int k = l; k < c->L; ++k) s *= c->opts.ns_growth;
  return s;
}

// One smoothing step on level l: u <- u + sum_s R_s^T W_s A_ss^{-1} R_s (f - A u).
// u_is_zero: u == 0 on entry (the residual is f; u is overwritten).
// r_ready: lev[l].r already holds f - A u.
template <typename T>
cudaError_t smooth_step(const mg_ctx* c, int l, T* u, const T* f, bool u_is_zero, bool r_ready) {
  cudaError_t e;
  const T* rin = f;
  if (!u_is_zero) {
    T* r = lvec<T>(c->lev[l].r);
    if (!r_ready) {
      ProfScope ps(c, kProfSipg, l);
      if ((e = launch_sipg<T>(c, l, u, f, r, 1)) != cudaSuccess) return e;
    }
    rin = r;
  }
  {
    ProfScope ps(c, kProfFdm, l);
    if ((e = launch_fdm<T>(c, l, rin)) != cudaSuccess) return e;
  }
  ProfScope ps(c, kProfScatter, l);
  return launch_scatter<T>(c, l, u, u_is_zero ? 0 : 1);
}

// Algorithm 1 (MultigridCycle).  uL, fL: fine-level vectors.
// u_zero: uL == 0 on entry; r_ready: lev[L].r == fL - A uL on entry.
template <typename T>
cudaError_t vcycle_t(const mg_ctx* c, T* uL, const T* fL, bool u_zero, bool r_ready) {
  const int L = c->L;
  T* u[kMaxLevels];
  const T* f[kMaxLevels];
  for (int l = 0; l <= L; ++l) {
    u[l] = (l == L) ? uL : lvec<T>(c->lev[l].u);
    f[l] = (l == L) ? fL : lvec<T>(c->lev[l].f);
  }
  cudaError_t e;
  for (int l = L; l >= 1; --l) {
    const int ns = steps_on_level(c, c->opts.ns_pre, l);
    const bool zero = (l < L) || u_zero;  // u_l <- 0 on the lower levels
    for (int st = 0; st < ns; ++st) {
      if ((e = smooth_step<T>(c, l, u[l], f[l], zero && st == 0, l == L && st == 0 && r_ready && !zero)) !=
          cudaSuccess)
        return e;
    }
    if (ns == 0 && zero && (e = launch_zero<T>(c, u[l], c->lev[l].N)) != cudaSuccess) return e;
    // f_{l-1} = I_l^T (f_l - A_l u_l)
    T* r = lvec<T>(c->lev[l].r);
    {
      ProfScope ps(c, kProfSipg, l);
      if ((e = launch_sipg<T>(c, l, u[l], f[l], r, 1)) != cudaSuccess) return e;
    }
    ProfScope ps(c, kProfRestrict, l);
    if ((e = launch_restrict<T>(c, l, r, lvec<T>(c->lev[l - 1].f))) != cudaSuccess) return e;
  }
  {
    ProfScope ps(c, kProfCoarse, 0);
    if ((e = coarse_solve_t<T>(c, f[0], u[0])) != cudaSuccess) return e;
  }
  for (int l = 1; l <= L; ++l) {
    {
      ProfScope ps(c, kProfProlong, l);
      if ((e = launch_prolong<T>(c, l, u[l - 1], u[l])) != cudaSuccess) return e;
    }
    const int ns = steps_on_level(c, c->opts.ns_post, l);
    for (int st = 0; st < ns; ++st)
      if ((e = smooth_step<T>(c, l, u[l], f[l], false, false)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// z = B r: one V-cycle from a zero guess, in FP64 or (mixed) in FP32 with the
// input scaled by 1/||r|| (kSlotRR must hold r.r).
cudaError_t precond(const mg_ctx* c, const double* r, double* z) {
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  if (c->opts.precision == MG_MIXED) {
    float* f32 = lvec<float>(c->lev[L].f);
    float* u32 = lvec<float>(c->lev[L].u);
    cudaError_t e;
    {
      ProfScope pv(c, kProfVector, L);
      if ((e = launch_to_f32(c, r, f32, N, kSlotRR)) != cudaSuccess) return e;
    }
    if ((e = vcycle_t<float>(c, u32, f32, true, false)) != cudaSuccess) return e;
    ProfScope pv(c, kProfVector, L);
    return launch_from_f32(c, u32, z, N, kSlotRR);
  }
  if (c->opts.precision == MG_DF64) {
    df64* fd = lvec<df64>(c->lev[L].f);
    df64* ud = lvec<df64>(c->lev[L].u);
    cudaError_t e;
    {
      ProfScope pv(c, kProfVector, L);
      if ((e = launch_split_df64(c, r, fd, N)) != cudaSuccess) return e;
    }
    if ((e = vcycle_t<df64>(c, ud, fd, true, false)) != cudaSuccess) return e;
    ProfScope pv(c, kProfVector, L);
    return launch_join_df64(c, ud, z, N, 0);
  }
  return vcycle_t<double>(c, z, r, true, false);
}

// FP32 smoother kernel per level.  fdm_tensor_cores = 1: the tensor-core
// kernel wherever the tiles fit it.  2: both kernels are timed on the level
// (CUDA events, a zero residual, after one warm-up launch each) and the
// faster one is kept.
cudaError_t choose_fdm_kernels(mg_ctx* c) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaSuccess;
  for (int l = 1; l <= c->L && e == cudaSuccess; ++l) {
    LevelInfo& lv = c->lev[l];
    lv.fdm_tc = 0;
    if (!fdm_tc_fits(c, l)) continue;
    if (c->opts.fdm_tensor_cores == 1) {
      lv.fdm_tc = 1;
      continue;
    }
    if (!e0 && ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)) break;
    float* r = lvec<float>(lv.r);
    if ((e = launch_zero<float>(c, r, lv.N)) != cudaSuccess) break;
    float best[2] = {0.f, 0.f};
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
      lv.fdm_tc = kind;
      if ((e = launch_fdm<float>(c, l, r)) != cudaSuccess) break;
      if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) break;
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = launch_fdm<float>(c, l, r);
      if (e != cudaSuccess || (e = cudaEventRecord(e1, c->stream)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      e = cudaEventElapsedTime(&best[kind], e0, e1);
    }
    lv.fdm_tc = (e == cudaSuccess && best[1] < best[0]) ? 1 : 0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

// Autotuner (mg_opts.autotune): on every level, time each kernel variant of
// the smoother, the operator and the scatter as the hierarchy's arithmetic
// runs them (CUDA events, one warm-up launch and three timed launches each,
// inputs zeroed), and keep the faster one per (kernel, level).
template <typename T>
cudaError_t autotune_levels_t(mg_ctx* c) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto timed = [&](auto&& run, float* ms) -> cudaError_t {
    cudaError_t er;
    if ((er = run()) != cudaSuccess) return er;
    if ((er = cudaEventRecord(e0, c->stream)) != cudaSuccess) return er;
    for (int k = 0; k < 3; ++k)
      if ((er = run()) != cudaSuccess) return er;
    if ((er = cudaEventRecord(e1, c->stream)) != cudaSuccess) return er;
    if ((er = cudaEventSynchronize(e1)) != cudaSuccess) return er;
    return cudaEventElapsedTime(ms, e0, e1);
  };
  for (int l = 1; l <= c->L && e == cudaSuccess; ++l) {
    LevelInfo& lv = c->lev[l];
    T* u = lvec<T>(lv.u);
    T* f = lvec<T>(lv.f);
    T* r = lvec<T>(lv.r);
    if ((e = launch_zero<T>(c, u, lv.N)) != cudaSuccess) break;
    if ((e = launch_zero<T>(c, f, lv.N)) != cudaSuccess) break;
    float t[3] = {0.f, 0.f, 0.f};
    if (std::is_same<T, float>::value && !lv.fdm_tc) {
      const int nv = fdm_c_applies(c, l) ? 3 : 2;
      int best = 0;
      for (int v = 0; v < nv && e == cudaSuccess; ++v) {
        lv.fdm_variant = v;
        e = timed([&]() { return launch_fdm<T>(c, l, f); }, &t[v]);
        if (t[v] < t[best]) best = v;
      }
      lv.fdm_variant = best;
    }
    if (!std::is_same<T, double>::value) {
      for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
        lv.sipg_plain = v;
        e = timed([&]() { return launch_sipg<T>(c, l, u, f, r, 1); }, &t[v]);
      }
      lv.sipg_plain = t[1] < t[0] ? 1 : 0;
    }
    for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
      lv.scatter_plain = v;
      e = timed([&]() { return launch_scatter<T>(c, l, u, 0); }, &t[v]);
    }
    lv.scatter_plain = t[1] < t[0] ? 1 : 0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

cudaError_t autotune_levels(mg_ctx* c) {
  if (c->opts.precision == MG_MIXED) return autotune_levels_t<float>(c);
  if (c->opts.precision == MG_DF64) return autotune_levels_t<df64>(c);
  return autotune_levels_t<double>(c);
}

// The first direction of the PCG iteration: z = B r projected to zero mean,
// p = z, rz = r . z (and p in double-float for the outer operator).
cudaError_t cg_start(const mg_ctx* c, double* r, double* z, double* p, df64* pdf) {
  const int64_t N = c->lev[c->L].N;
  cudaError_t e;
  if ((e = precond(c, r, z)) != cudaSuccess) return e;
  if ((e = launch_sum(c, z, N, kSlotSum)) != cudaSuccess) return e;
  if ((e = launch_sub_mean(c, z, N, kSlotSum)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(p, z, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) return e;
  if ((e = launch_dot(c, r, z, N, kSlotRZ)) != cudaSuccess) return e;
  if (pdf) e = launch_split_df64(c, p, pdf, N);
  return e;
}

// First half of a PCG iteration: q = A p (in double-float when pdf is given),
// alpha = rz / pq, x += alpha p, r -= alpha q, rr = |r - mean(r)|^2.  The mean
// of r (zero up to rounding: 1^T q = 0) is taken out where r is used, not
// stored.  Kernel launches only (no host synchronisation).
cudaError_t cg_step_a(const mg_ctx* c, double* x, double* p, double* r, double* q, df64* pdf, df64* qdf) {
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  cudaError_t e;
  if (pdf) {
    {
      ProfScope ps(c, kProfOuter, L);
      if ((e = launch_sipg<df64>(c, L, pdf, nullptr, qdf, 0)) != cudaSuccess) return e;
    }
    ProfScope pv(c, kProfVector, L);
    if ((e = launch_dot_dfq(c, p, qdf, q, N, kSlotPQ)) != cudaSuccess) return e;
  } else {
    {
      ProfScope ps(c, kProfOuter, L);
      if ((e = launch_sipg<double>(c, L, p, nullptr, q, 0)) != cudaSuccess) return e;
    }
    ProfScope pv(c, kProfVector, L);
    if ((e = launch_dot(c, p, q, N, kSlotPQ)) != cudaSuccess) return e;
  }
  ProfScope pv(c, kProfVector, L);
  return launch_cg_update(c, x, p, r, q, N);
}

// Second half: z = B r projected; beta = z_new . (r_new - r_old) / (z_old . r_old)
// = -alpha (z_new . q) / rz_old; p = z + beta p; rz = r . z.  Kernel launches only.
cudaError_t cg_step_b(const mg_ctx* c, double* p, double* r, double* q, double* z, df64* pdf) {
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  cudaError_t e;
  if (c->opts.precision == MG_MIXED) {
    float* f32 = lvec<float>(c->lev[L].f);
    float* u32 = lvec<float>(c->lev[L].u);
    {
      ProfScope pv(c, kProfVector, L);
      if ((e = launch_to_f32(c, r, f32, N, kSlotRR)) != cudaSuccess) return e;
    }
    if ((e = vcycle_t<float>(c, u32, f32, true, false)) != cudaSuccess) return e;
    ProfScope pv(c, kProfVector, L);
    return launch_cg_direction<float>(c, p, u32, q, r, N, pdf);
  }
  if (c->opts.precision == MG_DF64) {
    df64* fd = lvec<df64>(c->lev[L].f);
    df64* ud = lvec<df64>(c->lev[L].u);
    {
      ProfScope pv(c, kProfVector, L);
      if ((e = launch_split_df64(c, r, fd, N)) != cudaSuccess) return e;
    }
    if ((e = vcycle_t<df64>(c, ud, fd, true, false)) != cudaSuccess) return e;
    ProfScope pv(c, kProfVector, L);
    return launch_cg_direction<df64>(c, p, ud, q, r, N, pdf);
  }
  if ((e = vcycle_t<double>(c, z, r, true, false)) != cudaSuccess) return e;
  ProfScope pv(c, kProfVector, L);
  return launch_cg_direction<double>(c, p, z, q, r, N);
}

// ---- MG-CG with the outer iteration in double-float (mg_opts.outer_df64 = 2) ----
// The outer vectors live in the FP64 work vectors, reinterpreted as df64
// pairs: x in cg[7], r in cg[1], p in cg[3], q in cg[4], f in cg[0]; the
// FP32 preconditioner reads lev[L].f and writes lev[L].u.
bool outer_all_df64(const mg_ctx* c) { return c->opts.outer_df64 == 2 && c->opts.precision == MG_MIXED; }

struct OdfVecs {
  double* x64;
  df64 *x, *r, *p, *q;
  float *f32, *z32;
};

OdfVecs odf_vecs(const mg_ctx* c) {
  OdfVecs v;
  v.x64 = c->ws.cg[7];
  v.x = reinterpret_cast<df64*>(c->ws.cg[7]);
  v.r = reinterpret_cast<df64*>(c->ws.cg[1]);
  v.p = reinterpret_cast<df64*>(c->ws.cg[3]);
  v.q = reinterpret_cast<df64*>(c->ws.cg[4]);
  v.f32 = lvec<float>(c->lev[c->L].f);
  v.z32 = lvec<float>(c->lev[c->L].u);
  return v;
}

// The first direction: x (FP64, = u), f and r (FP64, zero mean, scal[Sum]
// its sum, scal[RR] its square norm) are split into pairs, q = 0, z = B r in
// FP32, p = z - mean(z), rz = z'.r'.  Launches only.
cudaError_t odf_start(const mg_ctx* c, const double* u, const double* f) {
  const int64_t N = c->lev[c->L].N;
  const OdfVecs v = odf_vecs(c);
  cudaError_t e;
  if ((e = launch_split_df64(c, f, reinterpret_cast<df64*>(c->ws.cg[0]), N)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(v.x64, u, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return e;
  if ((e = launch_odf_split(c, v.x64, N)) != cudaSuccess) return e;
  if ((e = launch_odf_split(c, c->ws.cg[1], N)) != cudaSuccess) return e;
  if ((e = launch_zero<double>(c, c->ws.cg[4], N)) != cudaSuccess) return e;
  if ((e = launch_odf_to_f32(c, v.r, v.f32, N)) != cudaSuccess) return e;
  if ((e = vcycle_t<float>(c, v.z32, v.f32, true, false)) != cudaSuccess) return e;
  return launch_odf_direction(c, v.p, v.z32, v.q, v.r, N, 1);
}

// q = A p; alpha; x, r updated; rr; the next preconditioner input.  Launches only.
cudaError_t odf_step_a(const mg_ctx* c) {
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  const OdfVecs v = odf_vecs(c);
  cudaError_t e;
  {
    ProfScope ps(c, kProfOuter, L);
    if ((e = launch_sipg<df64>(c, L, v.p, nullptr, v.q, 0)) != cudaSuccess) return e;
  }
  ProfScope pv(c, kProfVector, L);
  return launch_odf_update(c, v.x, v.p, v.r, v.q, v.f32, N);
}

// The true residual of the iterate (residual replacement): r = f - A x
// evaluated directly (double-float operator with compensated inner products:
// its error is a few 2^-48 of |f|, far below the tolerance), written over
// the recurrence residual, with scal[Sum], scal[RR] (|r - mean(r)|^2).
// Launches only.  The 48-bit recurrence residual drifts from the true one
// over many iterations (by about 7 % after 85), so convergence is confirmed
// on this residual, and a failed check continues from it (odf_replace).
cudaError_t odf_true_residual(const mg_ctx* c) {
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  const OdfVecs v = odf_vecs(c);
  cudaError_t e;
  if ((e = launch_sipg<df64>(c, L, v.x, reinterpret_cast<const df64*>(c->ws.cg[0]), v.r, 1)) != cudaSuccess)
    return e;
  return launch_odf_residual_norm(c, v.r, N);
}

// After a failed check: the next preconditioner input from the replaced
// residual.  Launches only.
cudaError_t odf_replace(const mg_ctx* c) {
  const OdfVecs v = odf_vecs(c);
  return launch_odf_to_f32(c, v.r, v.f32, c->lev[c->L].N);
}

// z = B r (FP32 V-cycle), beta, rz, p.  Launches only.
cudaError_t odf_step_b(const mg_ctx* c) {
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  const OdfVecs v = odf_vecs(c);
  cudaError_t e;
  if ((e = vcycle_t<float>(c, v.z32, v.f32, true, false)) != cudaSuccess) return e;
  ProfScope pv(c, kProfVector, L);
  return launch_odf_direction(c, v.p, v.z32, v.q, v.r, N, 0);
}

mg_status solve_impl(mg_ctx* c, double* u, const double* f, double tol, int maxit, int use_cg, int* iters,
                     double* relres, double* history) {
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  cudaError_t err;
  int it = 0;
  double r0 = 0.0, rn = 0.0;
  bool converged = false;
  if (!use_cg) {
    double* r = lvec<double>(c->lev[L].r);
    const bool mixed = c->opts.precision != MG_FP64;  // defect correction u += B r (B in FP32 or double-float)
    if (mixed) r = c->ws.cg[1];
    CK(launch_sipg<double>(c, L, u, f, r, 1));
    CK(launch_dot(c, r, r, N, kSlotRR));
    double rr = read_scalar(c, kSlotRR, &err);
    CK(err);
    r0 = rn = sqrt(rr);
    if (history) history[0] = r0;
    if (!std::isfinite(r0)) return fail(c, MG_EINVAL, "initial residual is not finite (NaN or Inf in u or f)");
    converged = r0 == 0.0;
    while (!converged && it < maxit) {
      ++it;
      // one cycle (FP64 V-cycle, or mixed defect correction u += B r) and the new residual norm
      CK(run_graph(c, kGraphMgCycle, u, f, [&]() -> cudaError_t {
        cudaError_t e;
        if (mixed) {
          double* z = c->ws.cg[2];
          if ((e = precond(c, r, z)) != cudaSuccess) return e;
          ProfScope pv(c, kProfVector, L);
          if ((e = launch_add(c, u, z, N)) != cudaSuccess) return e;
        } else if ((e = vcycle_t<double>(c, u, f, false, true)) != cudaSuccess) {
          return e;
        }
        {
          ProfScope ps(c, kProfOuter, L);
          if ((e = launch_sipg<double>(c, L, u, f, r, 1)) != cudaSuccess) return e;
        }
        ProfScope pv(c, kProfVector, L);
        return launch_dot(c, r, r, N, kSlotRR);
      }));
      double v = read_scalar(c, kSlotRR, &err);
      CK(err);
      rn = sqrt(v);
      if (history) history[it] = rn;
      if (!std::isfinite(rn)) return fail(c, MG_ENOCONV, "residual became non-finite");
      if (rn <= tol * r0) converged = true;
    }
  } else {
    double* x = u;
    double* r = c->ws.cg[1];
    double* z = c->ws.cg[2];
    double* p = c->ws.cg[3];
    double* q = c->ws.cg[4];
    const bool odf = outer_all_df64(c);
    CK(launch_sipg<double>(c, L, x, f, r, 1));
    CK(launch_sum(c, r, N, kSlotSum));
    CK(launch_sub_mean(c, r, N, kSlotSum));
    if (odf) CK(launch_sum(c, r, N, kSlotSum));  // sum(r) of the projected r, used by the first direction
    CK(launch_dot(c, r, r, N, kSlotRR));
    double rr = read_scalar(c, kSlotRR, &err);
    CK(err);
    r0 = rn = sqrt(rr);
    if (history) history[0] = r0;
    if (!std::isfinite(r0)) return fail(c, MG_EINVAL, "initial residual is not finite (NaN or Inf in u or f)");
    converged = r0 == 0.0;
    if (odf) {
      // the outer iteration in double-float pairs; x returns to u (FP64) at the end
      if (!converged) CK(odf_start(c, x, f));
      bool started = !converged;
      while (!converged && it < maxit) {
        ++it;
        CK(run_graph(c, kGraphOdfA, x, f, [&]() { return odf_step_a(c); }));
        double v = read_scalar(c, kSlotRR, &err);
        CK(err);
        rn = sqrt(v);
        if (history) history[it] = rn;
        if (!std::isfinite(rn)) return fail(c, MG_ENOCONV, "residual became non-finite");
        if (rn <= tol * r0) {
          // confirm on the true residual of the iterate
          CK(odf_true_residual(c));
          double t = read_scalar(c, kSlotRR, &err);
          CK(err);
          rn = sqrt(t);
          if (history) history[it] = rn;
          if (rn <= tol * r0) {
            converged = true;
            break;
          }
          CK(odf_replace(c));
        }
        CK(run_graph(c, kGraphOdfB, x, f, [&]() { return odf_step_b(c); }));
      }
      if (started) CK(launch_join_df64(c, reinterpret_cast<const df64*>(c->ws.cg[7]), x, N, 0));
    }
    // double-float copies of p and q for the outer operator (mg_opts.outer_df64), in the
    // smoother's correction buffer: written after each preconditioner, read before the next
    const bool df = c->opts.outer_df64 && c->opts.precision != MG_FP64;
    df64* pdf = df ? static_cast<df64*>(c->ws.corr) : nullptr;
    df64* qdf = df ? pdf + N : nullptr;
    if (!converged && !odf) CK(cg_start(c, r, z, p, pdf));
    while (!converged && !odf && it < maxit) {
      ++it;
      CK(run_graph(c, kGraphCgA, x, f, [&]() { return cg_step_a(c, x, p, r, q, pdf, qdf); }));
      double v = read_scalar(c, kSlotRR, &err);
      CK(err);
      rn = sqrt(v);
      if (history) history[it] = rn;
      if (!std::isfinite(rn)) return fail(c, MG_ENOCONV, "residual became non-finite");
      if (rn <= tol * r0) {
        converged = true;
        break;
      }
      CK(run_graph(c, kGraphCgB, x, f, [&]() { return cg_step_b(c, p, r, q, z, pdf); }));
    }
  }
  CK(launch_sum(c, u, N, kSlotSum));
  CK(launch_sub_mean(c, u, N, kSlotSum));
  int waits = 0;
  CK(cudaMemcpyAsync(&waits, c->ws.status + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (iters) *iters = it;
  if (waits != kDevOk) return fail(c, MG_ECUDA, "a tensor-core kernel gave up waiting for its MMAs");
  if (relres) *relres = r0 > 0.0 ? rn / r0 : 0.0;
  if (!converged) return fail(c, MG_ENOCONV, "maximum number of iterations reached");
  return MG_OK;
}

// Batched MG-CG (mg_solve_batch).  Every problem's launches are recorded and
// merged into grouped launches on the first problem's stream; host
// synchronisation once per iteration for all problems together.
struct BatchMember {
  mg_ctx* c;
  double *x, *r, *z, *p, *q;
  const double* f;
  df64 *pdf, *qdf;
  double r0 = 0.0, rn = 0.0;
  int it = 0;
  int status = MG_OK;
  bool active = true;
};

#ifndef MGDG_BATCH_CAPTURE_AFTER
#define MGDG_BATCH_CAPTURE_AFTER 5
#endif

// Recorded half iterations of a batch, keyed by the step and the set of
// active problems (it shrinks as problems converge): a sequence is recorded
// once, launched from the record while it is new, and captured as a CUDA
// graph when the same key occurs for the MGDG_BATCH_CAPTURE_AFTER-th time
// (0: never), so that short-lived sets do not pay for a capture.
struct BatchCache {
  struct Entry {
    uint64_t key;
    int uses;
    std::vector<LaunchRecorder> seqs;
    cudaGraphExec_t exec;
    long long nodes;  // kernel launches in the graph
  };
  cudaStream_t s = nullptr, cap = nullptr;
  std::vector<Entry> entries;
  ~BatchCache() {
    bool any = false;
    for (auto& e : entries) any = any || e.exec;
    if (any) cudaStreamSynchronize(s);
    for (auto& e : entries)
      if (e.exec) cudaGraphExecDestroy(e.exec);
    if (cap) cudaStreamDestroy(cap);
  }
};

cudaError_t capture_merged(BatchCache* bc, const std::vector<LaunchRecorder>& seqs, long long* launches,
                           cudaGraphExec_t* exec, int persist) {
  cudaError_t e;
  if (!bc->cap && (e = cudaStreamCreateWithFlags(&bc->cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = cudaStreamBeginCapture(bc->cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return e;
  const cudaError_t el = launch_merged(seqs, bc->cap, launches, persist);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(bc->cap, &graph);
  if (el != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return el != cudaSuccess ? el : ec;
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

// Record `step(member)` for every active member (or take the recorded
// sequences from the cache), then launch them merged.
template <typename F>
cudaError_t batch_step(std::vector<BatchMember>& ms, cudaStream_t s, long long* launches, F step,
                       BatchCache* cache = nullptr, int kind = 0) {
  uint64_t key = (uint64_t)kind << 32;
  const int persist = ms.empty() ? 0 : ms[0].c->opts.persistent;  // the first context's choice
  for (int i = 0; i < (int)ms.size(); ++i)
    if (ms[i].active) key |= 1ull << i;
  BatchCache::Entry* ent = nullptr;
  if (cache)
    for (auto& e : cache->entries)
      if (e.key == key) ent = &e;
  if (ent && ent->exec) {
    *launches += ent->nodes;
    return cudaGraphLaunch(ent->exec, s);
  }
  std::vector<LaunchRecorder> fresh;
  if (!ent) {
    fresh.reserve(ms.size());
    LaunchRecorder*& rec = launch_recorder();
    for (auto& m : ms) {
      if (!m.active) continue;
      fresh.emplace_back();
      rec = &fresh.back();
      const long long n0 = m.c->nlaunch;  // recorded, not launched for this context
      const cudaError_t e = step(m);
      m.c->nlaunch = n0;
      rec = nullptr;
      if (e != cudaSuccess) return e;
    }
    if (fresh.empty()) return cudaSuccess;
    if (!cache) return launch_merged(fresh, s, launches, persist);
    cache->entries.push_back({key, 0, std::move(fresh), nullptr, 0});
    ent = &cache->entries.back();
  }
  ent->uses += 1;
  if (MGDG_BATCH_CAPTURE_AFTER > 0 && ent->uses >= MGDG_BATCH_CAPTURE_AFTER) {
    const cudaError_t e = capture_merged(cache, ent->seqs, &ent->nodes, &ent->exec, persist);
    if (e != cudaSuccess) return e;
    *launches += ent->nodes;
    return cudaGraphLaunch(ent->exec, s);
  }
  return launch_merged(ent->seqs, s, launches, persist);
}

// Host copies of scalar slot `slot` of every active member (one gather
// launch, one copy, one synchronisation).
cudaError_t batch_read(std::vector<BatchMember>& ms, int slot, cudaStream_t s, std::vector<double>& out,
                       long long* launches) {
  const double* src[kMaxBatch];
  int idx[kMaxBatch], n = 0;
  for (int i = 0; i < (int)ms.size(); ++i)
    if (ms[i].active) {
      src[n] = ms[i].c->ws.scal + slot;
      idx[n++] = i;
    }
  out.assign(ms.size(), 0.0);
  if (n == 0) return cudaSuccess;
  double* dst = ms[0].c->ws.scal + kSlotBatch;
  double host[kMaxBatch];
  cudaError_t e;
  if ((e = launch_gather_scalars(src, n, dst, s)) != cudaSuccess) return e;
  ++*launches;
  if ((e = cudaMemcpyAsync(host, dst, n * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  for (int k = 0; k < n; ++k) out[idx[k]] = host[k];
  return cudaSuccess;
}

mg_status solve_batch_impl(std::vector<BatchMember>& ms, cudaStream_t s, double tol, int maxit, long long* launches,
                           std::string* err) {
  cudaError_t e;
  std::vector<double> v;
#define BCK(x)                                   \
  do {                                           \
    if ((e = (x)) != cudaSuccess) {              \
      *err = cudaGetErrorString(e);              \
      return MG_ECUDA;                           \
    }                                            \
  } while (0)
  // r = f - A x projected to zero mean, |r|
  BCK(batch_step(ms, s, launches, [&](BatchMember& m) -> cudaError_t {
    const int64_t N = m.c->lev[m.c->L].N;
    cudaError_t e2;
    if ((e2 = launch_sipg<double>(m.c, m.c->L, m.x, m.f, m.r, 1)) != cudaSuccess) return e2;
    if ((e2 = launch_sum(m.c, m.r, N, kSlotSum)) != cudaSuccess) return e2;
    if ((e2 = launch_sub_mean(m.c, m.r, N, kSlotSum)) != cudaSuccess) return e2;
    if (outer_all_df64(m.c) && (e2 = launch_sum(m.c, m.r, N, kSlotSum)) != cudaSuccess) return e2;
    return launch_dot(m.c, m.r, m.r, N, kSlotRR);
  }));
  BCK(batch_read(ms, kSlotRR, s, v, launches));
  for (int i = 0; i < (int)ms.size(); ++i) {
    BatchMember& m = ms[i];
    m.r0 = m.rn = sqrt(v[i]);
    if (!std::isfinite(m.r0)) {
      m.status = MG_EINVAL;
      m.active = false;
    } else if (m.r0 == 0.0) {
      m.active = false;
    }
  }
  // The cudaMemcpyAsync of cg_start is not a kernel: the first direction runs per problem.
  std::vector<bool> odf_started(ms.size(), false);
  for (int i = 0; i < (int)ms.size(); ++i) {
    BatchMember& m = ms[i];
    if (m.active) {
      const long long n0 = m.c->nlaunch;
      if (outer_all_df64(m.c)) {
        BCK(odf_start(m.c, m.x, m.f));
        odf_started[i] = true;
      } else {
        BCK(cg_start(m.c, m.r, m.z, m.p, m.pdf));
      }
      *launches += m.c->nlaunch - n0;
    }
  }
  BatchCache cache;
  cache.s = s;
  for (int it = 1; it <= maxit; ++it) {
    bool any = false;
    for (auto& m : ms) any = any || m.active;
    if (!any) break;
    BCK(batch_step(
        ms, s, launches,
        [&](BatchMember& m) {
          return outer_all_df64(m.c) ? odf_step_a(m.c) : cg_step_a(m.c, m.x, m.p, m.r, m.q, m.pdf, m.qdf);
        },
        &cache, 1));
    BCK(batch_read(ms, kSlotRR, s, v, launches));
    for (int i = 0; i < (int)ms.size(); ++i) {
      BatchMember& m = ms[i];
      if (!m.active) continue;
      m.it = it;
      m.rn = sqrt(v[i]);
      if (!std::isfinite(m.rn)) {
        m.status = MG_ENOCONV;
        m.active = false;
      } else if (m.rn <= tol * m.r0 && odf_started[i]) {
        // double-float recurrence: confirm on the FP64 residual (one problem at a time)
        const long long n0 = m.c->nlaunch;
        BCK(odf_true_residual(m.c));
        *launches += m.c->nlaunch - n0;
        std::vector<BatchMember> one(1, m);
        std::vector<double> t;
        BCK(batch_read(one, kSlotRR, s, t, launches));
        m.rn = sqrt(t[0]);
        if (m.rn <= tol * m.r0) {
          m.active = false;
        } else if (it == maxit) {
          m.status = MG_ENOCONV;
          m.active = false;
        } else {
          const long long n1 = m.c->nlaunch;
          BCK(odf_replace(m.c));
          *launches += m.c->nlaunch - n1;
        }
      } else if (m.rn <= tol * m.r0) {
        m.active = false;
      } else if (it == maxit) {
        m.status = MG_ENOCONV;
        m.active = false;
      }
    }
    BCK(batch_step(
        ms, s, launches,
        [&](BatchMember& m) { return outer_all_df64(m.c) ? odf_step_b(m.c) : cg_step_b(m.c, m.p, m.r, m.q, m.z, m.pdf); },
        &cache, 2));
  }
  // double-float iterates back to FP64, zero-mean solutions and the tensor-core wait flags
  for (int i = 0; i < (int)ms.size(); ++i)
    if (odf_started[i]) {
      BatchMember& m = ms[i];
      const int64_t N = m.c->lev[m.c->L].N;
      const long long n0 = m.c->nlaunch;
      BCK(launch_join_df64(m.c, reinterpret_cast<const df64*>(m.c->ws.cg[7]), m.x, N, 0));
      *launches += m.c->nlaunch - n0;
    }
  for (auto& m : ms) m.active = true;
  BCK(batch_step(ms, s, launches, [&](BatchMember& m) -> cudaError_t {
    const int64_t N = m.c->lev[m.c->L].N;
    cudaError_t e2;
    if ((e2 = launch_sum(m.c, m.x, N, kSlotSum)) != cudaSuccess) return e2;
    return launch_sub_mean(m.c, m.x, N, kSlotSum);
  }));
  std::vector<int> waits(ms.size(), 0);
  for (int i = 0; i < (int)ms.size(); ++i)
    BCK(cudaMemcpyAsync(&waits[i], ms[i].c->ws.status + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  for (int i = 0; i < (int)ms.size(); ++i)
    if (waits[i] != kDevOk && ms[i].status == MG_OK) ms[i].status = MG_ECUDA;
#undef BCK
  return MG_OK;
}

}  // namespace

extern "C" {

void mg_default_opts(mg_opts* o) {
  if (!o) return;
  o->overlap_mode = MG_OVERLAP_LAYERS;
  o->overlap_frac = 0.08;
  o->weight_profile = MG_WEIGHT_QUINTIC;
  o->ns_pre = 1;
  o->ns_post = 1;
  o->ns_growth = 1;
  o->precision = MG_FP64;
  o->fdm_tensor_cores = 0;
  o->outer_df64 = 0;
  o->stream = nullptr;
  o->weight_delta = MG_DELTA_DEFAULT;
  o->autotune = 0;
  o->fdm_operands = 0;
  o->persistent = 0;
}

mg_status mg_setup(double lx, double ly, double lz, int nx, int ny, int nz, int P, double penalty, int overlap,
                   const mg_opts* opts, mg_ctx** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (!(lx > 0 && ly > 0 && lz > 0) || nx < 3 || ny < 3 || nz < 3 || !(penalty > 0) || overlap < 0) return MG_EINVAL;
  if (nx > 512 || ny > 512 || nz > 512) return MG_EINVAL;  // coarse eigensolver pairs fit one block
  if (P < 2 || P > kMaxP || (P & (P - 1)) != 0) return MG_EINVAL;
  mg_opts o;
  mg_default_opts(&o);
  if (opts) o = *opts;
  if (o.ns_pre < 0 || o.ns_post < 0 || o.ns_growth < 1 || o.ns_pre + o.ns_post < 1) return MG_EINVAL;
  if (o.precision != MG_FP64 && o.precision != MG_MIXED && o.precision != MG_DF64) return MG_EINVAL;
  if (o.fdm_tensor_cores < 0 || o.fdm_tensor_cores > 2) return MG_EINVAL;
  if (o.outer_df64 < 0 || o.outer_df64 > 2) return MG_EINVAL;
  if (o.autotune < 0 || o.autotune > 1) return MG_EINVAL;
  if (o.fdm_operands < 0 || o.fdm_operands > 2) return MG_EINVAL;
  if (o.persistent < 0 || o.persistent > 2) return MG_EINVAL;
  if (o.weight_profile < MG_WEIGHT_QUINTIC || o.weight_profile > MG_WEIGHT_QUINTIC_NORMALISED) return MG_EINVAL;
  if (o.weight_delta < MG_DELTA_DEFAULT || o.weight_delta > MG_DELTA_STRIP) return MG_EINVAL;
  if (o.overlap_mode == MG_OVERLAP_LAYERS && o.weight_delta == MG_DELTA_STRIP) return MG_EINVAL;
  if (o.overlap_mode == MG_OVERLAP_MAX && o.weight_delta != MG_DELTA_DEFAULT) return MG_EINVAL;
  if (o.overlap_mode != MG_OVERLAP_LAYERS && o.overlap_mode != MG_OVERLAP_WIDTH && o.overlap_mode != MG_OVERLAP_MAX)
    return MG_EINVAL;
  if (o.overlap_mode == MG_OVERLAP_WIDTH && !(o.overlap_frac >= 0.0 && o.overlap_frac <= 0.5)) return MG_EINVAL;
  if (o.overlap_mode == MG_OVERLAP_MAX && !(o.overlap_frac >= 0.0 && o.overlap_frac <= 1.0)) return MG_EINVAL;
  if ((int64_t)nx * ny * nz > (int64_t)1 << 31) return MG_EINVAL;
  mg_ctx* c = new (std::nothrow) mg_ctx();
  if (!c) return MG_ENOMEM;
  c->len[0] = lx;
  c->len[1] = ly;
  c->len[2] = lz;
  c->ne[0] = nx;
  c->ne[1] = ny;
  c->ne[2] = nz;
  c->Ne = (int64_t)nx * ny * nz;
  c->P = P;
  c->L = 0;
  while ((1 << c->L) < P) ++c->L;
  c->penalty = penalty;
  c->overlap = overlap;
  c->opts = o;
  c->stream = static_cast<cudaStream_t>(o.stream);
  c->ready = false;
  for (int d = 0; d < 3; ++d) c->Ng[d] = 2 * c->ne[d];
  int64_t off = 0;
  auto tab = [&](int64_t count) {
    int64_t o2 = off;
    off += (count + 31) / 32 * 32;
    return o2;
  };
  for (int l = 0; l <= c->L; ++l) {
    LevelInfo& lv = c->lev[l];
    lv.P = 1 << l;
    lv.n = lv.P + 1;
    lv.N = c->Ne * (int64_t)lv.n * lv.n * lv.n;
    const double hmax = std::max(std::max(lx / nx, ly / ny), lz / nz);
    for (int d = 0; d < 3; ++d) {
      if (l == 0) {
        lv.no[d] = 0;
        lv.m[d] = 0;
        lv.delta[d] = 0.0;
        continue;
      }
      if (o.overlap_mode == MG_OVERLAP_MAX) {
        // strip of width min(frac max_j dx_j, dx_d): up to the whole neighbour element
        const double h = c->len[d] / c->ne[d];
        const double rel = std::min(o.overlap_frac * hmax, h) / h;
        lv.no[d] = layers_from_width(lv.P, rel);
        lv.delta[d] = 2.0 * rel;
        if (lv.no[d] == lv.n && c->ne[d] < 4) {
          delete c;
          return MG_EINVAL;
        }
      } else {
        const int maxno = lv.P / 2 + 1;
        const int no = (o.overlap_mode == MG_OVERLAP_LAYERS) ? overlap : layers_from_width(lv.P, o.overlap_frac);
        lv.no[d] = std::min(no, maxno);
        const bool strip = o.overlap_mode == MG_OVERLAP_WIDTH &&
                           (o.weight_delta == MG_DELTA_DEFAULT || o.weight_delta == MG_DELTA_STRIP);
        lv.delta[d] = strip ? std::min(2.0 * o.overlap_frac, 1.0)
                            : layer_delta(lv.P, lv.no[d], o.weight_delta == MG_DELTA_NODE ? MG_DELTA_NODE : MG_DELTA_MID);
      }
      lv.m[d] = lv.n + 2 * lv.no[d];
    }
    for (int d = 0; d < 3; ++d) {
      lv.h[d] = c->len[d] / c->ne[d];
      lv.g[d] = 2.0 / lv.h[d];
      lv.mu[d] = penalty * lv.P * (lv.P + 1.0) / (2.0 * lv.h[d]);
      DirTables& t = lv.t[d];
      t.nodes = tab(lv.n);
      t.weights = tab(lv.n);
      t.mass = tab(lv.n);
      t.lee = tab((int64_t)lv.n * lv.n);
      t.d0 = tab(lv.n);
      t.dp = tab(lv.n);
      t.ce = tab((int64_t)((lv.n + 1) / 2) * ((lv.n + 1) / 2));
      t.co = tab((int64_t)(lv.n / 2) * (lv.n / 2) + 1);
      t.fe = tab((lv.n + 1) / 2);
      t.fo = tab(lv.n / 2 + 1);
      t.fsc = tab(2);
      if (l >= 1) {
        t.S = tab((int64_t)lv.m[d] * lv.m[d]);
        t.SW = tab((int64_t)lv.m[d] * lv.m[d]);
        t.lam = tab(lv.m[d]);
        t.w = tab(lv.m[d]);
        t.Q = t.qlam = -1;
      } else {
        t.S = t.SW = t.lam = t.w = -1;
        t.Q = tab((int64_t)c->Ng[d] * c->Ng[d]);
        t.qlam = tab(c->Ng[d]);
      }
    }
    lv.dinv = (l >= 1) ? tab((int64_t)lv.m[0] * lv.m[1] * lv.m[2]) : -1;
    lv.dinvp = (l >= 1) ? tab((int64_t)lv.m[0] * ((lv.m[1] + 3) / 4 * 4) * ((lv.m[2] + 3) / 4 * 4)) : -1;
    lv.mass3 = tab((int64_t)lv.n * lv.n * lv.n);
    lv.J = (l >= 1) ? tab((int64_t)lv.n * (c->lev[l - 1].n)) : -1;
    lv.u = lv.f = lv.r = nullptr;
    lv.fdm_tc = 0;
    lv.fdm_variant = lv.sipg_plain = lv.scatter_plain = 0;
  }
  c->ws.tab_count = off;
  c->ws_bytes = make_layout(c).total;
  *out = c;
  return MG_OK;
}

mg_status mg_setup_graded(const double* hx, const double* hy, const double* hz, int nx, int ny, int nz, int P,
                          double penalty, int overlap, const mg_opts* opts, mg_ctx** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (!hx || !hy || !hz || nx < 3 || ny < 3 || nz < 3 || nx > 256 || ny > 256 || nz > 256) return MG_EINVAL;
  const double* hs[3] = {hx, hy, hz};
  const int ns[3] = {nx, ny, nz};
  double len[3];
  for (int d = 0; d < 3; ++d) {
    len[d] = 0.0;
    for (int e = 0; e < ns[d]; ++e) {
      if (!(hs[d][e] > 0.0) || !std::isfinite(hs[d][e])) return MG_EINVAL;
      len[d] += hs[d][e];
    }
  }
  mg_opts o;
  mg_default_opts(&o);
  if (opts) o = *opts;
  // graded meshes run the FP64 or the FP32 hierarchy (with the FP64 or the
  // double-float outer iteration) on node-layer overlaps, with the fixed kernels
  if (o.precision != MG_FP64 && o.precision != MG_MIXED) return MG_EINVAL;
  if (o.overlap_mode != MG_OVERLAP_LAYERS || o.fdm_tensor_cores != 0 || o.autotune != 0 || o.fdm_operands != 0)
    return MG_EINVAL;
  mg_ctx* c = nullptr;
  const mg_status st = mg_setup(len[0], len[1], len[2], nx, ny, nz, P, penalty, overlap, &o, &c);
  if (st != MG_OK) return st;
  c->graded = true;
  int64_t off = c->ws.tab_count;
  auto tab = [&](int64_t count) {
    int64_t o2 = off;
    off += (count + 31) / 32 * 32;
    return o2;
  };
  for (int d = 0; d < 3; ++d) {
    c->wid[d].assign(hs[d], hs[d] + ns[d]);
    c->org[d].assign(ns[d], 0.0);
    for (int e = 1; e < ns[d]; ++e) c->org[d][e] = c->org[d][e - 1] + c->wid[d][e - 1];
    c->gwid[d] = tab(ns[d]);
    c->gorg[d] = tab(ns[d]);
  }
  for (int l = 0; l <= c->L; ++l) {
    LevelInfo& lv = c->lev[l];
    for (int d = 0; d < 3; ++d) {
      DirTables& t = lv.t[d];
      const int64_t nd = ns[d], n = lv.n, m = lv.m[d];
      t.gblk = tab(nd * 3 * n * n);
      t.gmass = tab(nd * n);
      if (l >= 1) {
        t.gS = tab(nd * m * m);
        t.gSW = tab(nd * m * m);
        t.glam = tab(nd * m);
      }
    }
  }
  c->ws.tab_count = off;
  c->ws_bytes = make_layout(c).total;
  *out = c;
  return MG_OK;
}

mg_status mg_get_line_table(mg_ctx* c, int level, int dir, int line, int what, double* host_out, int capacity,
                            int* count) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!c->graded) return fail(c, MG_EINVAL, "not a graded mesh");
  if (!check_level(c, level, false) || dir < 0 || dir > 2 || line < 0 || line >= c->ne[dir] || !host_out || !count)
    return fail(c, MG_EINVAL, "bad arguments");
  const LevelInfo& lv = c->lev[level];
  const DirTables& t = lv.t[dir];
  const int64_t n = lv.n, m = lv.m[dir];
  int64_t off = -1, cnt = 0;
  switch (what) {
    case 0: off = t.gmass; cnt = n; break;
    case 1: off = t.gblk; cnt = 3 * n * n; break;
    case 2: off = t.glam; cnt = m; break;
    case 3: off = t.gS; cnt = m * m; break;
    default: return fail(c, MG_EINVAL, "unknown table");
  }
  if (off < 0) return fail(c, MG_EINVAL, "table not present on this level");
  if (cnt > capacity) return fail(c, MG_EINVAL, "capacity too small");
  CK(cudaMemcpyAsync(host_out, c->ws.tab64 + off + cnt * line, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *count = (int)cnt;
  return MG_OK;
}

int mg_is_graded(const mg_ctx* c) { return c && c->graded ? 1 : 0; }

mg_status mg_workspace_size(const mg_ctx* c, size_t* bytes) {
  if (!c || !bytes) return MG_EINVAL;
  *bytes = c->ws_bytes;
  return MG_OK;
}

mg_status mg_bind_workspace(mg_ctx* c, void* dptr, size_t bytes) {
  if (!c) return MG_EINVAL;
  if (!dptr || (reinterpret_cast<uintptr_t>(dptr) & 255) != 0) return fail(c, MG_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < c->ws_bytes) return fail(c, MG_ENOMEM, "workspace too small");
  Layout ly = make_layout(c);
  char* b = static_cast<char*>(dptr);
  Workspace& w = c->ws;
  w.base = b;
  w.bytes = bytes;
  w.tab64 = reinterpret_cast<double*>(b + ly.tab64);
  w.tab32 = reinterpret_cast<float*>(b + ly.tab32);
  w.tabdf = reinterpret_cast<df64*>(b + ly.tabdf);
  for (int l = 0; l <= c->L; ++l) {
    c->lev[l].u = b + ly.lev_u[l];
    c->lev[l].f = b + ly.lev_f[l];
    c->lev[l].r = b + ly.lev_r[l];
  }
  w.corr = b + ly.corr;
  w.coarse_a = reinterpret_cast<double*>(b + ly.ca);
  w.coarse_b = reinterpret_cast<double*>(b + ly.cb);
  w.coarse_f = reinterpret_cast<double*>(b + ly.cf);
  w.coarse_u = reinterpret_cast<double*>(b + ly.cu);
  for (int k = 0; k < 8; ++k) w.cg[k] = reinterpret_cast<double*>(b + ly.cg[k]);
  w.red = reinterpret_cast<double*>(b + ly.red);
  w.scal = reinterpret_cast<double*>(b + ly.scal);
  w.status = reinterpret_cast<int*>(b + ly.status);
  w.jac = reinterpret_cast<double*>(b + ly.jac);
  w.jac_count = ly.jac_count;
  w.gjac = c->graded ? reinterpret_cast<double*>(b + ly.gjac) : nullptr;
  w.gjac_line = ly.gjac_line;
  w.gjac_coarse = ly.gjac_coarse;
  CK(cudaMemsetAsync(w.status, 0, 256, c->stream));
  if (c->graded) {
    // element widths and left ends per direction, read by the setup kernels
    for (int d = 0; d < 3; ++d) {
      CK(cudaMemcpyAsync(w.tab64 + c->gwid[d], c->wid[d].data(), c->ne[d] * sizeof(double), cudaMemcpyHostToDevice,
                         c->stream));
      CK(cudaMemcpyAsync(w.tab64 + c->gorg[d], c->org[d].data(), c->ne[d] * sizeof(double), cudaMemcpyHostToDevice,
                         c->stream));
    }
  }
  CK(cudaMemsetAsync(w.scal, 0, kNumSlots * sizeof(double), c->stream));
  CK(launch_setup(c));
  int st = 0;
  CK(cudaMemcpyAsync(&st, w.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  c->tab32_host.assign(c->ws.tab_count, 0.0f);
  CK(cudaMemcpyAsync(c->tab32_host.data(), w.tab32, c->ws.tab_count * sizeof(float), cudaMemcpyDeviceToHost,
                     c->stream));
  c->tabdf_host.assign(c->ws.tab_count, df64(0.f, 0.f));
  CK(cudaMemcpyAsync(c->tabdf_host.data(), w.tabdf, c->ws.tab_count * sizeof(df64), cudaMemcpyDeviceToHost,
                     c->stream));
  // null mode of the coarse eigenbases: the smallest eigenvalue per direction
  for (int d = 0; d < 3; ++d) {
    std::vector<double> lam(c->Ng[d]);
    CK(cudaMemcpyAsync(lam.data(), w.tab64 + c->lev[0].t[d].qlam, lam.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->coarse_null[d] = (int)(std::min_element(lam.begin(), lam.end()) - lam.begin());
  }
  CK(cudaStreamSynchronize(c->stream));
  if (st != kDevOk) return fail(c, MG_ENOCONV, "setup eigensolver did not converge");
  if (c->opts.precision == MG_MIXED && !c->graded)  // graded meshes have their own smoother kernels
    for (int l = 1; l <= c->L; ++l) c->lev[l].fdm_variant = fdm_c_default_variant(c, l);
  if (c->opts.precision == MG_MIXED && c->opts.fdm_tensor_cores != 0) CK(choose_fdm_kernels(c));
  if (c->opts.autotune) {
    const long long n0 = c->nlaunch;
    CK(autotune_levels(c));
    CK(cudaStreamSynchronize(c->stream));
    c->nlaunch = n0;  // the trial launches are not the solver's
  }
  c->ready = true;
  return MG_OK;
}

int mg_num_levels(const mg_ctx* c) { return c ? c->L + 1 : 0; }

long long mg_num_dofs(const mg_ctx* c, int level) {
  if (!c || level < 0 || level > c->L) return -1;
  return c->lev[level].N;
}

int mg_level_layers(const mg_ctx* c, int level) { return mg_level_layers_dir(c, level, 0); }

mg_status mg_vcycle_df64(mg_ctx* c, double* u, const double* f) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (c->graded) return fail(c, MG_EINVAL, "the double-float multigrid is not built for graded meshes");
  if (!u || !f || u == f) return fail(c, MG_EINVAL, "null or aliased vector");
  const int L = c->L;
  const int64_t N = c->lev[L].N;
  df64* ud = reinterpret_cast<df64*>(c->ws.cg[5]);
  df64* fd = reinterpret_cast<df64*>(c->ws.cg[6]);
  CK(launch_split_df64(c, u, ud, N));
  CK(launch_split_df64(c, f, fd, N));
  CK(vcycle_t<df64>(c, ud, fd, false, false));
  CK(launch_join_df64(c, ud, u, N, 0));
  return MG_OK;
}

mg_status mg_smooth_df64(mg_ctx* c, int level, double* u, const double* f, int nsteps) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (c->graded) return fail(c, MG_EINVAL, "the double-float multigrid is not built for graded meshes");
  if (!check_level(c, level, true)) return MG_EINVAL;
  if (!u || !f || u == f || nsteps < 0) return fail(c, MG_EINVAL, "bad arguments");
  const int64_t N = c->lev[level].N;
  df64* ud = reinterpret_cast<df64*>(c->ws.cg[5]);
  df64* fd = reinterpret_cast<df64*>(c->ws.cg[6]);
  CK(launch_split_df64(c, u, ud, N));
  CK(launch_split_df64(c, f, fd, N));
  for (int k = 0; k < nsteps; ++k) CK(smooth_step<df64>(c, level, ud, fd, false, false));
  CK(launch_join_df64(c, ud, u, N, 0));
  return MG_OK;
}

mg_status mg_apply_sipg_df64(mg_ctx* c, int level, const double* u, double* Au) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, false)) return MG_EINVAL;
  if (!u || !Au || u == Au) return fail(c, MG_EINVAL, "null or aliased vector");
  const int64_t N = c->lev[level].N;
  df64* udf = static_cast<df64*>(c->ws.corr);
  df64* adf = udf + N;
  if ((int64_t)(2 * N) > c->lev[c->L].N * 2) return fail(c, MG_EINVAL, "level too large for the scratch");
  CK(launch_split_df64(c, u, udf, N));
  CK(launch_sipg<df64>(c, level, udf, nullptr, adf, 0));
  CK(launch_dot_dfq(c, u, adf, Au, N, kSlotSum));
  return MG_OK;
}

mg_status mg_selftest_bounded_wait(mg_ctx* c, int level, int* timed_out) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!timed_out || c->opts.precision != MG_MIXED || level < 1 || level > c->L || !fdm_tc_fits(c, level))
    return fail(c, MG_EINVAL, "the level cannot run the tensor-core smoother");
  *timed_out = 0;
  float* r = lvec<float>(c->lev[level].r);
  CK(launch_zero<float>(c, r, c->lev[level].N));
  CK(launch_fdm_tc(c, level, r, 1));
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->ws.status + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemsetAsync(c->ws.status + 1, 0, sizeof(int), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *timed_out = st == kDevTimeout ? 1 : 0;
  return MG_OK;
}

int mg_level_kernel_variant(const mg_ctx* c, int level, int kind) {
  if (!c || level < 1 || level > c->L) return -1;
  const LevelInfo& lv = c->lev[level];
  switch (kind) {
    case 0: return lv.fdm_variant;
    case 1: return lv.sipg_plain;
    case 2: return lv.scatter_plain;
    default: return -1;
  }
}

int mg_level_fdm_tensor_cores(const mg_ctx* c, int level) {
  if (!c || level < 0 || level > c->L) return -1;
  return c->lev[level].fdm_tc;
}

int mg_level_layers_dir(const mg_ctx* c, int level, int dir) {
  if (!c || level < 0 || level > c->L || dir < 0 || dir > 2) return -1;
  return c->lev[level].no[dir];
}

mg_status mg_node_coords(mg_ctx* c, int level, double* x, double* y, double* z) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, false)) return MG_EINVAL;
  if (!x || !y || !z) return fail(c, MG_EINVAL, "null pointer");
  CK(launch_coords(c, level, x, y, z));
  return MG_OK;
}

mg_status mg_rhs(mg_ctx* c, const double* f, double* b) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!f || !b || f == b) return fail(c, MG_EINVAL, "bad pointers");
  CK(launch_rhs(c, f, b));
  return MG_OK;
}

mg_status mg_apply_sipg(mg_ctx* c, int level, const double* u, double* Au) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, false)) return MG_EINVAL;
  if (!u || !Au || u == Au) return fail(c, MG_EINVAL, "bad pointers");
  CK(launch_sipg<double>(c, level, u, nullptr, Au, 0));
  return MG_OK;
}

mg_status mg_apply_sipg_f32(mg_ctx* c, int level, const float* u, float* Au) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, false)) return MG_EINVAL;
  if (!u || !Au || u == Au) return fail(c, MG_EINVAL, "bad pointers");
  CK(launch_sipg<float>(c, level, u, nullptr, Au, 0));
  return MG_OK;
}

mg_status mg_residual(mg_ctx* c, int level, const double* u, const double* f, double* r) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, false)) return MG_EINVAL;
  if (!u || !f || !r || r == u || r == f) return fail(c, MG_EINVAL, "bad pointers");
  CK(launch_sipg<double>(c, level, u, f, r, 1));
  return MG_OK;
}

mg_status mg_smooth(mg_ctx* c, int level, double* u, const double* f, int nsteps) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, true)) return MG_EINVAL;
  if (!u || !f || u == f || nsteps < 0) return fail(c, MG_EINVAL, "bad arguments");
  for (int k = 0; k < nsteps; ++k) CK(smooth_step<double>(c, level, u, f, false, false));
  return MG_OK;
}

mg_status mg_smooth_f32(mg_ctx* c, int level, float* u, const float* f, int nsteps) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, true)) return MG_EINVAL;
  if (!u || !f || u == f || nsteps < 0) return fail(c, MG_EINVAL, "bad arguments");
  for (int k = 0; k < nsteps; ++k) CK(smooth_step<float>(c, level, u, f, false, false));
  return MG_OK;
}

mg_status mg_restrict_residual(mg_ctx* c, int level, const double* u, const double* f, double* fc) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, true)) return MG_EINVAL;
  if (!u || !f || !fc) return fail(c, MG_EINVAL, "null pointer");
  double* r = lvec<double>(c->lev[level].r);
  CK(launch_sipg<double>(c, level, u, f, r, 1));
  CK(launch_restrict<double>(c, level, r, fc));
  return MG_OK;
}

mg_status mg_prolongate(mg_ctx* c, int level, const double* uc, double* u) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, true)) return MG_EINVAL;
  if (!uc || !u) return fail(c, MG_EINVAL, "null pointer");
  CK(launch_prolong<double>(c, level, uc, u));
  return MG_OK;
}

mg_status mg_coarse_solve(mg_ctx* c, const double* f0, double* u0) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!f0 || !u0 || f0 == u0) return fail(c, MG_EINVAL, "bad pointers");
  CK(launch_coarse_solve(c, f0, u0));
  return MG_OK;
}

mg_status mg_vcycle(mg_ctx* c, double* u, const double* f) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!u || !f || u == f) return fail(c, MG_EINVAL, "bad pointers");
  CK(run_graph(c, kGraphVcycle, u, f, [&]() { return vcycle_t<double>(c, u, f, false, false); }));
  return MG_OK;
}

mg_status mg_vcycle_f32(mg_ctx* c, float* u, const float* f) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!u || !f || u == f) return fail(c, MG_EINVAL, "bad pointers");
  CK(run_graph(c, kGraphVcycle32, u, f, [&]() { return vcycle_t<float>(c, u, f, false, false); }));
  return MG_OK;
}

mg_status mg_solve(mg_ctx* c, double* u, const double* f, double tol, int maxit, int use_cg, int* iters,
                   double* relres, double* history) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!u || !f || u == f || maxit < 0 || !(tol >= 0.0)) return fail(c, MG_EINVAL, "bad arguments");
  NvtxRange range(use_cg ? "mg_solve MG-CG" : "mg_solve MG");
  return solve_impl(c, u, f, tol, maxit, use_cg ? 1 : 0, iters, relres, history);
}

mg_status mg_solve_host(mg_ctx* c, double* u_host, const double* f_host, double tol, int maxit, int use_cg,
                        int* iters, double* relres, double* history) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!u_host || !f_host || maxit < 0 || !(tol >= 0.0)) return fail(c, MG_EINVAL, "bad arguments");
  const int64_t N = c->lev[c->L].N;
  double* u = c->ws.cg[5];
  double* f = c->ws.cg[6];
  CK(cudaMemcpyAsync(f, f_host, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(u, u_host, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  mg_status st = solve_impl(c, u, f, tol, maxit, use_cg ? 1 : 0, iters, relres, history);
  if (st != MG_OK && st != MG_ENOCONV) return st;
  CK(cudaMemcpyAsync(u_host, u, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return st;
}

mg_status mg_get_table(mg_ctx* c, int level, int dir, int what, double* host_out, int capacity, int* count) {
  mg_status s = need_ready(c);
  if (s != MG_OK) return s;
  if (!check_level(c, level, false) || dir < 0 || dir > 2 || !host_out || !count)
    return fail(c, MG_EINVAL, "bad arguments");
  const LevelInfo& lv = c->lev[level];
  const DirTables& t = lv.t[dir];
  int64_t off = -1, cnt = 0;
  const int n = lv.n, m = lv.m[dir], Ng = c->Ng[dir];
  switch (what) {
    case 0: off = t.nodes; cnt = n; break;
    case 1: off = t.weights; cnt = n; break;
    case 2: off = t.mass; cnt = n; break;
    case 3: off = t.lee; cnt = (int64_t)n * n; break;
    case 4: off = t.lam; cnt = m; break;
    case 5: off = t.S; cnt = (int64_t)m * m; break;
    case 6: off = t.w; cnt = m; break;
    case 7: off = lv.J; cnt = level >= 1 ? (int64_t)n * c->lev[level - 1].n : 0; break;
    case 8: off = t.qlam; cnt = Ng; break;
    case 9: off = t.Q; cnt = (int64_t)Ng * Ng; break;
    default: return fail(c, MG_EINVAL, "unknown table");
  }
  if (off < 0 || cnt <= 0) return fail(c, MG_EINVAL, "table not present on this level");
  if (cnt > capacity) return fail(c, MG_EINVAL, "capacity too small");
  CK(cudaMemcpyAsync(host_out, c->ws.tab64 + off, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *count = (int)cnt;
  return MG_OK;
}

mg_status mg_solve_batch(mg_ctx* const* ctxs, int count, double* const* u, const double* const* f, double tol,
                         int maxit, int* iters, double* relres, int* status) {
  if (!ctxs || !u || !f || count < 1 || count > kMaxBatch || !(tol > 0.0) || maxit < 1) return MG_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || !u[i] || !f[i]) return MG_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[0], MG_EINVAL, "a context appears twice in the batch");
    if (!ctxs[i]->ready) return fail(ctxs[0], MG_ENOTREADY, "workspace not bound");
    if (ctxs[i]->graded) return fail(ctxs[0], MG_EINVAL, "graded meshes are solved one at a time");
  }
  mg_ctx* c0 = ctxs[0];
  const cudaStream_t s = c0->stream;
  std::vector<BatchMember> ms(count);
  std::vector<cudaStream_t> saved(count);
  std::vector<bool> prof(count);
  for (int i = 0; i < count; ++i) {
    mg_ctx* c = ctxs[i];
    const int64_t N = c->lev[c->L].N;
    BatchMember& m = ms[i];
    m.c = c;
    m.x = u[i];
    m.f = f[i];
    m.r = c->ws.cg[1];
    m.z = c->ws.cg[2];
    m.p = c->ws.cg[3];
    m.q = c->ws.cg[4];
    const bool df = c->opts.outer_df64 && c->opts.precision != MG_FP64;
    m.pdf = df ? static_cast<df64*>(c->ws.corr) : nullptr;
    m.qdf = df ? m.pdf + N : nullptr;
    saved[i] = c->stream;
    prof[i] = c->prof_on;
    c->stream = s;  // every launch of the batch goes to the first problem's stream
    c->prof_on = false;
  }
  std::string err;
  long long launches = 0;
  mg_status st;
  {
    NvtxRange range("mg_solve_batch");
    st = solve_batch_impl(ms, s, tol, maxit, &launches, &err);
  }
  for (int i = 0; i < count; ++i) {
    ctxs[i]->stream = saved[i];
    ctxs[i]->prof_on = prof[i];
    if (iters) iters[i] = ms[i].it;
    if (relres) relres[i] = ms[i].r0 > 0.0 ? ms[i].rn / ms[i].r0 : 0.0;
    if (status) status[i] = st != MG_OK ? st : ms[i].status;
  }
  c0->batch_launches += launches;
  if (st != MG_OK) return fail(c0, st, err);
  return MG_OK;
}

const char* mg_last_error(const mg_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

long long mg_batch_launches(const mg_ctx* c) { return c ? c->batch_launches : -1; }

long long mg_kernel_launches(const mg_ctx* c) { return c ? c->nlaunch : -1; }

mg_status mg_profile(mg_ctx* c, int enable) {
  if (!c) return MG_EINVAL;
  c->prof_on = enable != 0;
  if (enable) c->prof_used = 0;
  return MG_OK;
}

mg_status mg_profile_result(mg_ctx* c, int kind, int level, double* total_ms, long long* count) {
  if (!c || !total_ms || !count || kind < 0 || kind >= kProfKinds) return MG_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  long long n = 0;
  for (size_t i = 0; i < c->prof_used; ++i) {
    const mg_ctx::ProfRec& r = c->prof[i];
    if (r.kind != kind || (level >= 0 && r.level != level)) continue;
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *count = n;
  return MG_OK;
}

void mg_destroy(mg_ctx* c) {
  if (!c) return;
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto& r : c->prof) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  delete c;
}

}  // extern "C"
