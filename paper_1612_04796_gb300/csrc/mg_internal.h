// Internal declarations of the GB300 multigrid library: context, device table
// layout and the host-side launchers of every kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <cuda/std/tuple>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mgdg.h"
#include "df64.cuh"

namespace mgdg {

// Programmatic dependent launch.  Hot-path kernels are launched with
// launch_pdl, which lets a kernel be launched as soon as the blocks of its
// predecessor in the stream (or graph) have exited, before that grid has
// formally completed; every such kernel starts with pdl_entry(), which waits
// until the predecessor has completed and its writes are visible, before
// touching memory.  (Triggering the successor early, at the start of each
// kernel, was measured slower: its waiting blocks compete for the SMs.)  A
// kernel launched without the attribute passes the wait at once.
__device__ __forceinline__ void pdl_entry() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- batched execution: kernel bodies, grouped launches, launch recording ----
//
// A kernel body is a __device__ function that takes the block index and the
// number of blocks it may assume (BlockIdx) in place of blockIdx.x and
// gridDim.x.  Its plain kernel passes the real ones; its grouped twin
// (k_grouped) runs the bodies of several independent problems in one launch:
// the launch's blocks are split into consecutive ranges, one per problem,
// each range running the body with that problem's parameters and its own
// block numbering, as the plain kernel would (same per-block work, same
// reduction order).
struct BlockIdx {
  int b, g;  // block index, number of blocks
};
__device__ __forceinline__ BlockIdx plain_block() { return BlockIdx{(int)blockIdx.x, (int)gridDim.x}; }

#ifndef MGDG_MAX_BATCH
#define MGDG_MAX_BATCH 16
#endif
constexpr int kMaxBatch = MGDG_MAX_BATCH;  // problems per grouped launch

template <typename A>
struct Grouped {
  int count;
  int start[kMaxBatch + 1];  // first block of each problem; start[count] = the launch's blocks
  A a[kMaxBatch];            // each problem's kernel parameters
};

template <int LB, auto Body, typename... Ps>
__global__ void __launch_bounds__(LB) k_grouped(const __grid_constant__ Grouped<cuda::std::tuple<Ps...>> g) {
  pdl_entry();
  int r = 0;
  while (r + 1 < g.count && (int)blockIdx.x >= g.start[r + 1]) ++r;
  const BlockIdx bi{(int)blockIdx.x - g.start[r], g.start[r + 1] - g.start[r]};
  cuda::std::apply([&](const Ps&... ps) { Body(bi, ps...); }, g.a[r]);
}

// Persistent form of the grouped twin: at most as many blocks as the SMs
// hold at once, each looping over the launch's virtual blocks (the problem
// ranges of k_grouped, in increasing order), with a block barrier between two
// virtual blocks because the bodies reuse their shared memory.  Every virtual
// block does the work of the same block of k_grouped.  (No body returns
// before a barrier of its own, so every thread reaches the loop's barrier.)
template <int LB, auto Body, typename... Ps>
__global__ void __launch_bounds__(LB) k_grouped_p(const __grid_constant__ Grouped<cuda::std::tuple<Ps...>> g) {
  pdl_entry();
  const int total = g.start[g.count];
  int r = 0;
  for (int vb = (int)blockIdx.x; vb < total; vb += (int)gridDim.x) {
    while (r + 1 < g.count && vb >= g.start[r + 1]) ++r;
    const BlockIdx bi{vb - g.start[r], g.start[r + 1] - g.start[r]};
    cuda::std::apply([&](const Ps&... ps) { Body(bi, ps...); }, g.a[r]);
    __syncthreads();
  }
}

// Persistent grouped launches (mg_opts.persistent): 0 = where the launch has
// more blocks than the GPU holds at once, 1 = always, 2 = never.
enum PersistMode : int { kPersistAuto = 0, kPersistAlways = 1, kPersistNever = 2 };

// One recorded launch: the plain kernel (its identity), the launch shape, its
// parameters packed as cuda::std::tuple<kernel parameter types...>, how to
// replay it alone and (if the kernel has a body) how to launch the grouped
// twin for several records of the same kernel.
struct LaunchRec {
  const void* key = nullptr;
  dim3 grid, block;
  size_t smem = 0;
  std::vector<unsigned char> args;
  cudaError_t (*plain)(const LaunchRec&, cudaStream_t) = nullptr;
  cudaError_t (*grouped)(const LaunchRec* const*, int, cudaStream_t, int persist) = nullptr;
};

// While a host thread has a recorder installed, launch_pdl appends to it
// instead of launching (batched execution, batch.cu).
struct LaunchRecorder {
  std::vector<LaunchRec> recs;
};
LaunchRecorder*& launch_recorder();

inline cudaError_t launch_pdl_now(const void* kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, kernel, args);
}

template <typename... KArgs>
cudaError_t launch_tuple(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         cuda::std::tuple<KArgs...>& t) {
  void* ptrs[sizeof...(KArgs) > 0 ? sizeof...(KArgs) : 1];
  int i = 0;
  cuda::std::apply([&](KArgs&... v) { ((ptrs[i++] = (void*)&v), ...); }, t);
  return launch_pdl_now((const void*)kernel, grid, block, smem, s, ptrs);
}

template <typename... KArgs>
cudaError_t replay_plain(const LaunchRec& r, cudaStream_t s) {
  using Tup = cuda::std::tuple<KArgs...>;
  Tup t;
  memcpy((void*)&t, r.args.data(), sizeof(Tup));
  return launch_tuple(reinterpret_cast<void (*)(KArgs...)>(const_cast<void*>(r.key)), r.grid, r.block, r.smem, s,
                      t);
}

// Launch the grouped twin of Body for n problems: parameter sets a[i] (each
// a cuda::std::tuple<KArgs...>) with grid[i] blocks each.
// Allow `kernel` `smem` bytes of dynamic shared memory (once per kernel and size).
inline cudaError_t allow_smem(const void* kernel, size_t smem, std::atomic<size_t>& smem_set) {
  if (smem <= smem_set.load()) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  size_t cur = smem_set.load();
  while (cur < smem && !smem_set.compare_exchange_weak(cur, smem)) {
  }
  return cudaSuccess;
}

template <int LB, auto Body, typename... KArgs>
cudaError_t launch_twin(const void* const* a, const unsigned* grid, int n, dim3 block, size_t smem, cudaStream_t s,
                        int persist = kPersistAuto) {
  using Tup = cuda::std::tuple<KArgs...>;
  Grouped<Tup> g;
  g.count = n;
  g.start[0] = 0;
  for (int i = 0; i < n; ++i) {
    memcpy((void*)&g.a[i], a[i], sizeof(Tup));
    g.start[i + 1] = g.start[i] + (int)grid[i];
  }
  const int total = g.start[n];
  void* ptrs[1] = {(void*)&g};
  if (persist != kPersistNever) {
    auto* ptwin = k_grouped_p<LB, Body, KArgs...>;
    static std::atomic<size_t> psmem_set{48 * 1024};
    cudaError_t e = allow_smem((const void*)ptwin, smem, psmem_set);
    if (e != cudaSuccess) return e;
    // resident blocks per SM at this block size and shared memory (the largest
    // size asked for so far; a block count for fewer bytes is a lower bound)
    static std::atomic<long long> occ_key{-1};
    static std::atomic<int> occ_val{0};
    const long long key = (long long)block.x * (1LL << 32) + (long long)smem;
    int per_sm = occ_key.load() == key ? occ_val.load() : 0;
    if (per_sm == 0) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ptwin, (int)block.x, smem)) != cudaSuccess)
        return e;
      per_sm = per_sm > 0 ? per_sm : 1;
      occ_val.store(per_sm);
      occ_key.store(key);
    }
    const int resident = 152 * per_sm;
    if (persist == kPersistAlways || total > resident)
      return launch_pdl_now((const void*)ptwin, dim3(total < resident ? total : resident), block, smem, s, ptrs);
  }
  auto* twin = k_grouped<LB, Body, KArgs...>;
  static std::atomic<size_t> smem_set{48 * 1024};  // dynamic shared memory the twin is allowed so far
  const cudaError_t e = allow_smem((const void*)twin, smem, smem_set);
  if (e != cudaSuccess) return e;
  return launch_pdl_now((const void*)twin, dim3(total), block, smem, s, ptrs);
}

template <int LB, auto Body, typename... KArgs>
cudaError_t launch_grouped(const LaunchRec* const* r, int n, cudaStream_t s, int persist) {
  const void* a[kMaxBatch];
  unsigned grid[kMaxBatch];
  for (int i = 0; i < n; ++i) {
    a[i] = r[i]->args.data();
    grid[i] = r[i]->grid.x;
  }
  return launch_twin<LB, Body, KArgs...>(a, grid, n, r[0]->block, r[0]->smem, s, persist);
}

// Launch `kernel` with programmatic dependent launch, or record it while a
// recorder is installed (LaunchRecorder).  Body (optional, may be a null
// pointer): the kernel's body; a recorded launch of a kernel with a body is
// later run by the body's grouped twin k_grouped (with LB as launch bounds),
// together with other problems' launches of the same kernel.  The twin is a
// separate compilation of the body (it may contract multiply-adds
// differently from the plain kernel), so batched solves agree with single
// solves to rounding, and bit for bit with each other whatever the batch.
template <auto Body = nullptr, int LB = 256, typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cuda::std::tuple<KArgs...> t(static_cast<KArgs>(args)...);
  LaunchRecorder* rec = launch_recorder();
  if (!rec) return launch_tuple(kernel, grid, block, smem, s, t);
  LaunchRec r;
  r.key = (const void*)kernel;
  r.grid = grid;
  r.block = block;
  r.smem = smem;
  r.plain = &replay_plain<KArgs...>;
  if constexpr (Body != nullptr) {
    if (grid.y == 1 && grid.z == 1) r.grouped = &launch_grouped<LB, Body, KArgs...>;
  }
  r.args.resize(sizeof(t));
  memcpy(r.args.data(), (const void*)&t, sizeof(t));
  rec->recs.push_back(std::move(r));
  return cudaSuccess;
}

// Arithmetic types whose kernels have grouped twins: all of them (batched
// solves merge the launches of the FP64, FP32 and double-float hierarchies
// and of the vector passes).
template <typename T>
constexpr bool kTwinType = true;

constexpr int kMaxLevels = 6;   // P <= 32
constexpr int kMaxP = 32;
constexpr int kMaxN = kMaxP + 1;        // nodes per element and direction
constexpr int kMaxM = 3 * kMaxN;         // widest subdomain line (strips of whole neighbour elements)
constexpr int kRedBlocks = 1216;        // largest grid of the two-stage reductions (8 per SM)

// Slots of the device scalar array ws.scal.
enum Slot : int {
  kSlotRZ = 0,      // r . z
  kSlotPQ = 1,      // p . q
  kSlotAlpha = 2,   // alpha
  kSlotZQ = 3,      // z . q
  kSlotRR = 4,      // r . r
  kSlotSum = 5,     // scratch sum for mean projections
  kSlotMassF = 6,   // sum M f
  kSlotMass = 7,    // sum M
  kSlotScale = 8,   // norm used to scale FP32 preconditioner input
  kSlotBeta = 9,    // CG beta
  kSlotMuZ = 10,    // mean of the preconditioned residual z
  kSlotBatch = 16,  // 16 .. 16 + kMaxBatch - 1: scalars gathered from a batch's problems
  kSlotCoarse = 60, // coarse-solve mean
  kNumSlots = 64
};

// Status word written by device code (setup eigensolvers) and read by the host.
// Word 0: setup eigensolvers; word 1: bounded waits of the tensor-core kernels.
enum DevStatus : int { kDevOk = 0, kDevNoConv = 1, kDevTimeout = 2 };

// Offsets (in values) of the 1D tables of one level and direction inside the
// table arrays tab64 / tab32 (same offsets in both).
struct DirTables {
  int64_t nodes, weights, mass, lee, d0, dp;  // n, n, n, n*n, n, n
  // even/odd form of M^{-1} L_ee (ne = (n+1)/2, no = n/2): ce ne*ne, co no*no,
  // face vectors fe (ne), fo (no) and the scalars fsc = {mu / m_0, g / (2 m_0)}
  int64_t ce, co, fe, fo, fsc;
  int64_t S, SW, lam, w;                      // m*m, m*m, m, m  (level >= 1)
  int64_t Q, qlam;                            // Ng*Ng, Ng       (level 0)
  // Graded meshes (-1 on uniform ones), per element line e of this direction
  // (n_d lines): gblk + 3 n^2 e: the rows of element e of the 1D matrix L,
  // blocks L[e][e-1], L[e][e], L[e][e+1] (n x n, row-major); gmass + n e:
  // (h_e / 2) w; level >= 1: gS / gSW + m^2 e, glam + m e: the eigenbasis of
  // the subdomain line centred on element e (SW with the weights folded in).
  int64_t gblk = -1, gmass = -1, gS = -1, gSW = -1, glam = -1;
};

struct LevelInfo {
  int P, n;              // order, nodes per direction
  int m[3], no[3];       // subdomain width and overlap layers per direction
  double delta[3];       // hat-weight half-width per direction (reference units, <= 2)
  int64_t N;             // DOFs
  double h[3], g[3], mu[3];
  DirTables t[3];
  int64_t dinv;          // m_x m_y m_z: 1 / (lam_x[a] + lam_y[b] + lam_z[c])
  int64_t dinvp;         // the same values at (b + ru4(m_y) a) ru4(m_z) + c, zero padded
                         // (ru4 = rounded up to a multiple of 4; tensor-core smoother)
  int64_t mass3;         // n^3: mass_x[i] mass_y[j] mass_z[k]
  int fdm_tc;            // FP32 smoother contractions on the tensor cores (1) or CUDA cores (0)
  // Kernel variants of single solves (mg_opts.autotune picks them by timing):
  // fdm_variant 0 = the FP32 smoother k_fdm_c, 1 = the shared-memory k_fdm_m,
  // 2 = k_fdm_c's passes split over three grid-wide kernels (the default on
  // cubic levels with m >= 11); 1 = the plain
  // operator k_sipg_n instead of k_sipg_c; the scatter k_scatter_n2 instead of
  // the element-aligned k_scatter_e.
  int fdm_variant, sipg_plain, scatter_plain;
  int64_t J;             // n * n_c interpolation from level l-1 (level >= 1)
  // device vectors (bytes sized for FP64; FP32 code uses the first half)
  void* u;
  void* f;
  void* r;
};

struct Workspace {
  char* base = nullptr;
  size_t bytes = 0;
  double* tab64 = nullptr;
  float* tab32 = nullptr;
  df64* tabdf = nullptr;       // the FP64 tables split into double-float pairs
  int64_t tab_count = 0;
  void* corr = nullptr;        // smoother corrections, Ne * m_x m_y m_z (largest level)
  double* coarse_a = nullptr;  // coarse FDM scratch, N_0 each
  double* coarse_b = nullptr;
  double* coarse_f = nullptr;  // FP64 coarse rhs / solution for the FP32 hierarchy
  double* coarse_u = nullptr;
  double* cg[8] = {nullptr};   // FP64 outer vectors: x, r, z, p, q, u_io, f_io, spare
  double* red = nullptr;       // reduction partials (up to 8 columns of kRedBlocks)
  double* scal = nullptr;      // device scalars (64)
  int* status = nullptr;       // device status word
  double* jac = nullptr;       // eigensolver scratch
  int64_t jac_count = 0;
  double* gjac = nullptr;      // graded meshes: eigensolver scratch of the element lines
  int64_t gjac_line = 0, gjac_coarse = 0;  // doubles per line block, per coarse block
};

}  // namespace mgdg

struct mg_ctx {
  double len[3];
  int ne[3];
  int64_t Ne;
  int P, L;
  double penalty;
  int overlap;
  mg_opts opts;
  cudaStream_t stream;
  mgdg::LevelInfo lev[mgdg::kMaxLevels];
  int Ng[3];               // coarse 1D sizes 2 n_d
  int coarse_null[3];      // index of the constant eigenvector per direction
  // Graded mesh (mg_setup_graded): element widths per direction, and the
  // table offsets of the widths and of the elements' left ends.
  bool graded = false;
  std::vector<double> wid[3], org[3];
  int64_t gwid[3] = {-1, -1, -1}, gorg[3] = {-1, -1, -1};
  mgdg::Workspace ws;
  size_t ws_bytes;
  bool ready;
  std::string err;
  // instrumentation: kernel launch count and optional per-group CUDA events
  // (mutable: the launchers take a const context)
  struct ProfRec {
    int kind, level;
    cudaEvent_t a, b;
  };
  mutable long long nlaunch = 0;
  long long batch_launches = 0;  // launches of batched solves led by this context
  // CUDA graphs of recurring launch sequences (V-cycle, CG steps), keyed by
  // kind and the two vector pointers they were captured with.
  struct GraphEntry {
    int kind;
    const void* a;
    const void* b;
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  bool use_graphs = true;
  std::vector<float> tab32_host;  // host copies of the FP32 and double-float tables (kernel parameters
  std::vector<mgdg::df64> tabdf_host;  // of the FP32 smoother and the FP32 / double-float operators)
  mutable bool prof_on = false;
  mutable std::vector<ProfRec> prof;
  mutable size_t prof_used = 0;
};

namespace mgdg {

// Kernel groups timed by the profiler (mg_profile_result kinds).
// kProfSipg: the level operators inside the V-cycle; kProfOuter: the outer
// iteration's fine-level residual or q = A p (FP64 or double-float);
// kProfVector: the outer iteration's vector passes (inner products, updates,
// mean projections, FP64 <-> FP32 / double-float conversions).
enum ProfKind : int { kProfFdm = 0, kProfScatter, kProfSipg, kProfRestrict, kProfProlong, kProfCoarse, kProfVector,
                      kProfOuter, kProfKinds };

// ---- batched execution (batch.cu) ----
// Launch the recorded sequences of several problems on stream s, merged into
// grouped launches; *launches += the number of launches made.
cudaError_t launch_merged(const std::vector<LaunchRecorder>& seqs, cudaStream_t s, long long* launches,
                          int persist);
// out[i] = *src[i] (device scalars of up to kMaxBatch problems), one launch.
cudaError_t launch_gather_scalars(const double* const* src, int n, double* out, cudaStream_t s);

// ---- setup (setup.cu) ----
cudaError_t launch_setup(mg_ctx* c);

// Level-0 tables only (three blocks), explicit pointers; used by the
// allocation-free coarse solve (noalloc.cu).
cudaError_t launch_setup_coarse_tables(const double len[3], const int ne[3], double penalty, double* tab,
                                       const DirTables t[3], double* scratch, int64_t per_block, int* status,
                                       cudaStream_t s);

// ---- graded meshes (setup.cu, graded.cu) ----
// Tables of the element lines of every level and the graded coarse eigenbases.
cudaError_t launch_setup_graded(mg_ctx* c);
// out = A u (residual 0) or f - A u on level l from the per-line blocks.
template <typename T>
cudaError_t launch_gsipg(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual);
// Subdomain corrections (gather + fast diagonalisation with per-line
// eigenbases) into ws.corr, in the layout of launch_fdm.
template <typename T>
cudaError_t launch_gfdm(const mg_ctx* c, int l, const T* r);
// The same with compile-time widths (graded_fdm.cu): cubic odd m <= 25;
// cudaErrorNotSupported otherwise.
template <typename T>
cudaError_t launch_gfdm_fixed(const mg_ctx* c, int l, const T* r);
// u0 -= mean(u0) on level 0 (on a graded mesh the coarse solve's M-orthonormal
// eigenbases give a solution whose Euclidean mean is not zero).
template <typename T>
cudaError_t launch_gmean_zero(const mg_ctx* c, T* u0);
// out = f0 - mean(f0) in FP64 (level 0): the projection onto the range of A_0.
template <typename T>
cudaError_t launch_gcenter(const mg_ctx* c, const T* f0, double* out);
cudaError_t launch_grhs(const mg_ctx* c, const double* f, double* b);
cudaError_t launch_gcoords(const mg_ctx* c, int l, double* x, double* y, double* z);

// ---- operator (sipg_kernels.cuh, instantiated in sipg_f64.cu / sipg_f32.cu / sipg_df64.cu) ----
// out = mode==0 ? A u : f - A u, on level l, T = double | float.
template <typename T>
cudaError_t launch_sipg(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual);  // T: double, float, df64
// FP32 / double-float operator with shared-memory element blocks and the
// coefficients as kernel parameters (sipg_const.cu): orders 2, 4, 8, 16 on
// meshes that give every SM a block; cudaErrorNotSupported otherwise.
cudaError_t launch_sipg_c(const mg_ctx* c, int l, const float* u, const float* f, float* out, int residual);
cudaError_t launch_sipg_c(const mg_ctx* c, int l, const df64* u, const df64* f, df64* out, int residual);

// ---- smoother (schwarz.cu) ----
// Corrections of all subdomains from residual r into ws.corr, then
// u = beta*u + scatter(corr).  beta is 0 (u := correction) or 1.
template <typename T>
cudaError_t launch_fdm(const mg_ctx* c, int l, const T* r);
template <typename T>
cudaError_t launch_scatter(const mg_ctx* c, int l, T* u, int accumulate);
// FP32 corrections on the tensor cores (fdm_tc.cu); cudaErrorNotSupported if
// the level's subdomain tiles do not fit the kernel's shared/tensor memory.
// self_test = 1: no MMA is issued and nothing arrives on the barrier, so the
// kernel's first (shortened) wait runs out and it reports kDevTimeout.
cudaError_t launch_fdm_tc(const mg_ctx* c, int l, const float* r, int self_test = 0);
bool fdm_tc_fits(const mg_ctx* c, int l);
// FP32 corrections with the 1D factors as kernel parameters (fdm_const.cu):
// cubic odd widths 3..35; cudaErrorNotSupported otherwise.
cudaError_t launch_fdm_c(const mg_ctx* c, int l, const float* r);  // k_fdm_c, or split if fdm_variant == 2
bool fdm_c_applies(const mg_ctx* c, int l);
int fdm_c_default_variant(const mg_ctx* c, int l);  // 2 on cubic levels with m >= 11, else 0

// ---- transfers (transfer.cu) ----
template <typename T>
cudaError_t launch_restrict(const mg_ctx* c, int l, const T* r_fine, T* f_coarse);
template <typename T>
cudaError_t launch_prolong(const mg_ctx* c, int l, const T* u_coarse, T* u_fine);

// ---- coarse solve (coarse.cu) ----
cudaError_t launch_coarse_solve(const mg_ctx* c, const double* f0, double* u0);
cudaError_t launch_coarse_solve_f32(const mg_ctx* c, const float* f0, float* u0);
cudaError_t launch_coarse_solve_df64(const mg_ctx* c, const df64* f0, df64* u0);
// The six fast-diagonalisation passes of the coarse solve with explicit
// pointers; f0's mean is read from scal[mean_slot] (sum of f0).
cudaError_t launch_coarse_fdm_raw(const double* const Q[3], const double* const lam[3], const int Ng[3],
                                  const int ne[3], const int null_mode[3], const double* f0, double* A, double* B,
                                  double* u0, const double* scal, int mean_slot, cudaStream_t s);

// ---- vectors (blas.cu) ----
// dot products: result into device scalar slot `slot` of ws.scal
cudaError_t launch_dot(const mg_ctx* c, const double* x, const double* y, int64_t n, int slot);
cudaError_t launch_sum(const mg_ctx* c, const double* x, int64_t n, int slot);
cudaError_t launch_sub_mean(const mg_ctx* c, double* x, int64_t n, int sum_slot);
// Fused CG steps (one pass each plus a one-block finish):
//  cg_update: alpha = scal[RZ] / scal[PQ]; x += alpha p; r -= alpha q;
//             scal[Sum] = sum r, scal[RR] = |r - mean(r)|^2.
//  cg_direction: z = zscale * zsrc (zscale = sqrt(scal[RR]) for an FP32 z, else 1);
//             with z' = z - mean(z), r' = r - mean(r) (sum r in scal[Sum]) and
//             q of zero sum (1^T A = 0): beta = -alpha z'.q / scal[RZ];
//             scal[RZ] = z'.r'; p = z' + beta p.
cudaError_t launch_cg_update(const mg_ctx* c, double* x, const double* p, double* r, const double* q, int64_t n);
template <typename TZ>
cudaError_t launch_cg_direction(const mg_ctx* c, double* p, const TZ* z, const double* q, const double* r, int64_t n,
                                df64* pdf = nullptr);
// Double-float support of the outer operator: y = x split into pairs; and
// q = to_double(qdf) with scal[slot] = p . q in the same pass.
cudaError_t launch_split_df64(const mg_ctx* c, const double* x, df64* y, int64_t n);
cudaError_t launch_join_df64(const mg_ctx* c, const df64* x, double* y, int64_t n, int accumulate);
cudaError_t launch_dot_dfq(const mg_ctx* c, const double* p, const df64* qdf, double* q, int64_t n, int slot);
cudaError_t launch_add(const mg_ctx* c, double* y, const double* x, int64_t n);  // y += x
// Blocks of the two-stage reductions for n values, and their second stages
// over ws.red: the sum of one column into scal[slot]; the CG update's two
// columns into scal[Sum] and scal[RR] (|r - mean(r)|^2).
int reduction_blocks(int64_t n);
cudaError_t launch_final_sum(const mg_ctx* c, int nb, int slot);
cudaError_t launch_update_final(const mg_ctx* c, int nb, int64_t n);

// ---- outer MG-CG in double-float arithmetic (blas_df.cu; mg_opts.outer_df64 = 2) ----
// Vectors x, r, p, q stored as df64 pairs, z the FP32 preconditioner output.
//  update: pq = p . q; alpha = rz / pq; x += alpha p; r -= alpha q;
//          scal[Sum], scal[RR] of the new r; r32 = r / sqrt(rr_old), scal[Scale] = sqrt(rr_old).
//  direction: with z' = Scale z - mean: beta = -alpha z'.q / rz (0 if first);
//          rz = z'.r'; p = z' + beta p (p = z' if first).
cudaError_t launch_odf_update(const mg_ctx* c, df64* x, const df64* p, df64* r, const df64* q, float* r32,
                              int64_t n);
cudaError_t launch_odf_direction(const mg_ctx* c, df64* p, const float* z, const df64* q, const df64* r, int64_t n,
                                 int first);
cudaError_t launch_odf_split(const mg_ctx* c, double* v, int64_t n);  // FP64 -> df64, in place
// scal[Sum] = sum r, scal[RR] = |r - mean(r)|^2 of a double-float vector
cudaError_t launch_odf_residual_norm(const mg_ctx* c, const df64* r, int64_t n);
// y = r / sqrt(scal[RR]) (FP32), scal[Scale] = sqrt(scal[RR])
cudaError_t launch_odf_to_f32(const mg_ctx* c, const df64* r, float* y, int64_t n);
cudaError_t launch_to_f32(const mg_ctx* c, const double* x, float* y, int64_t n, int norm_slot);
cudaError_t launch_from_f32(const mg_ctx* c, const float* x, double* y, int64_t n, int norm_slot);
cudaError_t launch_rhs(const mg_ctx* c, const double* f, double* b);
cudaError_t launch_coords(const mg_ctx* c, int l, double* x, double* y, double* z);
template <typename T>
cudaError_t launch_zero(const mg_ctx* c, T* x, int64_t n);

}  // namespace mgdg
