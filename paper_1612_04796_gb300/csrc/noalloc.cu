// Allocation-free coarse solve: mg_coarse_solve_noalloc.
//
// Callers that may not allocate device memory -- for example a plugin that a
// host framework hands only its input and output buffers because the
// framework owns all device memory, or a latency-critical path that cannot
// accept the implicit device synchronisation of an allocation -- cannot
// provide the workspace that mg_bind_workspace needs.  This entry point
// computes u0 = A_0^+ f0 on the P_0 = 1 level from the mesh parameters alone:
// its scratch (the three coarse eigenbases, the eigensolver work space, two
// work vectors and the reduction slots) is the file-scope device array below,
// which every GPU that loads the library holds until the process exits.  The
// caller passes only f0 and u0.
//
// The array's name in host code is a host-side stand-in, not a device
// address; the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <math.h>

#include <mutex>

#include "mg_internal.h"

namespace mgdg {
namespace {

constexpr int kNaMaxElems = 32;                                        // per direction
constexpr int kNaMaxNg = 2 * kNaMaxElems;                              // coarse line size
constexpr int64_t kNaMaxN0 = 8LL * kNaMaxElems * kNaMaxElems * kNaMaxElems;  // 262,144 coarse DOFs
// Layout of the array (in doubles).
constexpr int64_t kNaSmall = 32;                                       // padded 1D table of <= 2 values
constexpr int64_t kNaTabPerDir = 6 * kNaSmall + kNaMaxNg * kNaMaxNg + kNaMaxNg;
constexpr int64_t kNaJacPerBlock = 4LL * kNaMaxNg * kNaMaxNg + 4 * kNaMaxNg + 64;
constexpr int64_t kNaTab = 0;
constexpr int64_t kNaJac = kNaTab + 3 * kNaTabPerDir;
constexpr int64_t kNaA = kNaJac + 3 * kNaJacPerBlock;
constexpr int64_t kNaB = kNaA + kNaMaxN0;
constexpr int64_t kNaScal = kNaB + kNaMaxN0;                           // 2 sums
constexpr int64_t kNaStatus = kNaScal + 8;                             // int status word
constexpr int64_t kNaCount = 589824;                                   // 4.5 MiB
static_assert(kNaStatus + 8 <= kNaCount, "scratch layout exceeds the array");

__device__ __align__(256) double g_na_scratch[kNaCount];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_addr[kNaMaxDevices] = {nullptr};

// Device address of g_na_scratch on the current device (looked up once per device).
cudaError_t scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (g_na_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = static_cast<double*>(p);
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

// Deterministic single-block sum of x[0..n) into *out.
__global__ void __launch_bounds__(1024) k_na_sum(const double* __restrict__ x, int64_t n, double* out) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_na_sub_mean(double* x, int64_t n, const double* sum) {
  const double mean = *sum / (double)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] -= mean;
}

}  // namespace
}  // namespace mgdg

using namespace mgdg;

extern "C" mg_status mg_coarse_solve_noalloc(double lx, double ly, double lz, int nx, int ny, int nz, double penalty,
                                             const double* f0, double* u0, void* stream) {
  if (!(lx > 0 && ly > 0 && lz > 0) || !(penalty > 0) || !f0 || !u0 || f0 == u0) return MG_EINVAL;
  if (nx < 3 || ny < 3 || nz < 3 || nx > kNaMaxElems || ny > kNaMaxElems || nz > kNaMaxElems) return MG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return MG_ECUDA;
  const double len[3] = {lx, ly, lz};
  const int ne[3] = {nx, ny, nz};
  int Ng[3];
  DirTables t[3];
  for (int d = 0; d < 3; ++d) {
    Ng[d] = 2 * ne[d];
    const int64_t o = kNaTab + d * kNaTabPerDir;
    t[d].nodes = o;
    t[d].weights = o + kNaSmall;
    t[d].mass = o + 2 * kNaSmall;
    t[d].lee = o + 3 * kNaSmall;
    t[d].d0 = o + 4 * kNaSmall;
    t[d].dp = o + 5 * kNaSmall;
    t[d].Q = o + 6 * kNaSmall;
    t[d].qlam = o + 6 * kNaSmall + (int64_t)kNaMaxNg * kNaMaxNg;
    t[d].S = t[d].SW = t[d].lam = t[d].w = -1;
    t[d].ce = t[d].co = t[d].fe = t[d].fo = t[d].fsc = -1;
  }
  double* tab = base + kNaTab;
  double* scal = base + kNaScal;
  int* status = reinterpret_cast<int*>(base + kNaStatus);
  const int64_t N0 = 8LL * nx * ny * nz;
  // The array keeps the previous call's contents: the status word must start at zero.
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return MG_ECUDA;
  if (launch_setup_coarse_tables(len, ne, penalty, tab, t, base + kNaJac, kNaJacPerBlock, status, s) != cudaSuccess)
    return MG_ECUDA;
  // null mode = the smallest eigenvalue of each periodic line (the constants)
  double lam[3][kNaMaxNg];
  int st = 0;
  for (int d = 0; d < 3; ++d)
    if (cudaMemcpyAsync(lam[d], tab + t[d].qlam, Ng[d] * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return MG_ECUDA;
  if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MG_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MG_ECUDA;
  if (st != kDevOk) return MG_ENOCONV;
  int null_mode[3];
  for (int d = 0; d < 3; ++d) {
    int best = 0;
    for (int k = 1; k < Ng[d]; ++k)
      if (lam[d][k] < lam[d][best]) best = k;
    null_mode[d] = best;
  }
  const double* Q[3] = {tab + t[0].Q, tab + t[1].Q, tab + t[2].Q};
  const double* L[3] = {tab + t[0].qlam, tab + t[1].qlam, tab + t[2].qlam};
  k_na_sum<<<1, 1024, 0, s>>>(f0, N0, scal);
  if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
  if (launch_coarse_fdm_raw(Q, L, Ng, ne, null_mode, f0, base + kNaA, base + kNaB, u0, scal, 0, s) != cudaSuccess)
    return MG_ECUDA;
  k_na_sum<<<1, 1024, 0, s>>>(u0, N0, scal + 1);
  int blocks = (int)((N0 + 255) / 256);
  k_na_sub_mean<<<blocks, 256, 0, s>>>(u0, N0, scal + 1);
  if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
  return MG_OK;
}
