// Vector kernels of the outer iteration and helpers (FP64 unless noted):
// inner products and sums with a fixed two-stage reduction order (so repeated
// runs give identical bits), the CG updates of the inexact preconditioned CG
// (Section 3.2) with their scalars kept on the device, mean projections onto
// the range of the singular periodic operator, FP64 <-> FP32 conversions with
// scaling for the FP32 preconditioner, the weak right-hand side b = M f
// (Section 2, GLL quadrature) and the node coordinates.
#include "mg_internal.h"

namespace mgdg {
namespace {

constexpr int kThreads = 256;

__device__ double block_reduce(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  return sh[0];
}

// mode 0: sum x*y   mode 1: sum x   (T = double | float input)
template <typename T>
__device__ __forceinline__ void partial_body(BlockIdx bi_, const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                             int mode, double* partial) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    acc += mode == 0 ? (double)x[i] * (double)y[i] : (double)x[i];
  double r = block_reduce(acc, sh);
  if (threadIdx.x == 0) partial[bi_.b] = r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_partial(const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                  int mode, double* partial) {
  pdl_entry();
  partial_body<T>(plain_block(), x, y, n, mode, partial);
}

__device__ __forceinline__ void final_body(BlockIdx bi_, const double* partial, int nb, double* scal, int slot) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
  double r = block_reduce(acc, sh);
  if (threadIdx.x == 0) scal[slot] = r;
}

__global__ void __launch_bounds__(kThreads) k_final(const double* partial, int nb, double* scal, int slot) {
  pdl_entry();
  final_body(plain_block(), partial, nb, scal, slot);
}

// Scalars that every thread needs are formed once per block (thread 0,
// shared memory): on this part a per-thread FP64 division or square root
// costs as much FP64-pipe time as the pass's per-element arithmetic.
template <typename T>
__device__ __forceinline__ void sub_mean_body(BlockIdx bi_, T* x, int64_t n, const double* scal, int slot) {
  __shared__ double s_mean;
  if (threadIdx.x == 0) s_mean = scal[slot] / (double)n;
  __syncthreads();
  const T mean = (T)s_mean;
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    x[i] -= mean;
}

template <typename T>
__global__ void k_sub_mean(T* x, int64_t n, const double* scal, int slot) {
  pdl_entry();
  sub_mean_body<T>(plain_block(), x, n, scal, slot);
}

// The CG update with the partial sums of the new r and r^2 (columns 0, 1).
__device__ __forceinline__ void cg_update_body(BlockIdx bi_, double* __restrict__ x, const double* __restrict__ p,
                                               double* __restrict__ r, const double* __restrict__ q, int64_t n,
                                               double* scal, double* partial) {
  __shared__ double sh[kThreads];
  __shared__ double s_alpha;
  if (threadIdx.x == 0) {
    s_alpha = scal[kSlotRZ] / scal[kSlotPQ];
    if (bi_.b == 0) scal[kSlotAlpha] = s_alpha;
  }
  __syncthreads();
  const double alpha = s_alpha;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s1 += ri;
    s2 += ri * ri;
  }
  const double b1 = block_reduce(s1, sh);
  __syncthreads();
  const double b2 = block_reduce(s2, sh);
  if (threadIdx.x == 0) {
    partial[bi_.b] = b1;
    partial[bi_.g + bi_.b] = b2;
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_update(double* __restrict__ x, const double* __restrict__ p,
                                  double* __restrict__ r, const double* __restrict__ q, int64_t n, double* scal,
                                  double* partial) {
  pdl_entry();
  cg_update_body(plain_block(), x, p, r, q, n, scal, partial);
}

// Sum `cols` columns of nb partials each, in a fixed order, into v[0 .. cols).
__device__ void final_columns(const double* partial, int nb, int cols, double* v, double* sh) {
  for (int k = 0; k < cols; ++k) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[k * nb + i];
    v[k] = block_reduce(acc, sh);
    __syncthreads();
  }
}

__device__ __forceinline__ void cg_update_final_body(BlockIdx bi_, const double* partial, int nb, double* scal,
                                                     int64_t n) {
  __shared__ double sh[kThreads];
  double v[2];
  final_columns(partial, nb, 2, v, sh);
  if (threadIdx.x == 0) {
    scal[kSlotSum] = v[0];
    scal[kSlotRR] = fmax(v[1] - v[0] * v[0] / (double)n, 0.0);
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_update_final(const double* partial, int nb, double* scal, int64_t n) {
  pdl_entry();
  cg_update_final_body(plain_block(), partial, nb, scal, n);
}

template <typename TZ>
__device__ __forceinline__ double z_scale(const double* scal) {
  if (sizeof(TZ) == sizeof(double)) return 1.0;
  const double nrm = sqrt(scal[kSlotRR]);
  return nrm > 0.0 ? nrm : 1.0;
}

// Partial sums of z, z.q, z.r (columns 0 .. 2), z taken unscaled (the FP32
// preconditioner's scale is applied to the totals).
template <typename TZ>
__device__ __forceinline__ void cg_sums_body(BlockIdx bi_, const TZ* __restrict__ zs, const double* __restrict__ q,
                                             const double* __restrict__ r, int64_t n, double* partial) {
  __shared__ double sh[kThreads];
  double a[3] = {0.0, 0.0, 0.0};
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x) {
    const double z = (double)zs[i];
    a[0] += z;
    a[1] += z * q[i];
    a[2] += z * r[i];
  }
  for (int k = 0; k < 3; ++k) {
    const double b = block_reduce(a[k], sh);
    __syncthreads();
    if (threadIdx.x == 0) partial[k * bi_.g + bi_.b] = b;
  }
}

template <typename TZ>
__global__ void __launch_bounds__(kThreads) k_cg_sums(const TZ* __restrict__ zs, const double* __restrict__ q,
                                  const double* __restrict__ r, int64_t n, double* partial) {
  pdl_entry();
  cg_sums_body<TZ>(plain_block(), zs, q, r, n, partial);
}

// With z' = z - mean(z): z'.q' = z.q (1^T q = 1^T A p = 0) and
// z'.r' = z.r - sum(z) sum(r) / n (sum(r) from the update pass).
template <typename TZ>
__device__ __forceinline__ void cg_sums_final_body(BlockIdx bi_, const double* partial, int nb, double* scal,
                                                   int64_t n) {
  __shared__ double sh[kThreads];
  double v[3];
  final_columns(partial, nb, 3, v, sh);
  if (threadIdx.x == 0) {
    const double zsc = z_scale<TZ>(scal), inv = 1.0 / (double)n;
    const double sz = zsc * v[0], zq = zsc * v[1];
    const double zr = zsc * v[2] - sz * scal[kSlotSum] * inv;
    scal[kSlotZQ] = zq;
    scal[kSlotBeta] = -scal[kSlotAlpha] * zq / scal[kSlotRZ];
    scal[kSlotMuZ] = sz * inv;
    scal[kSlotRZ] = zr;
  }
}

template <typename TZ>
__global__ void __launch_bounds__(kThreads) k_cg_sums_final(const double* partial, int nb, double* scal, int64_t n) {
  pdl_entry();
  cg_sums_final_body<TZ>(plain_block(), partial, nb, scal, n);
}

// p = (z - mean(z)) + beta p; pdf (if given) receives p split into double-float pairs
template <typename TZ>
__device__ __forceinline__ void cg_newdir_body(BlockIdx bi_, double* __restrict__ p, const TZ* __restrict__ zs,
                                               int64_t n, const double* scal, df64* __restrict__ pdf) {
  __shared__ double s_zsc;
  if (threadIdx.x == 0) s_zsc = z_scale<TZ>(scal);
  __syncthreads();
  const double zsc = s_zsc, muz = scal[kSlotMuZ], beta = scal[kSlotBeta];
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x) {
    const double v = ((double)zs[i] * zsc - muz) + beta * p[i];
    p[i] = v;
    if (pdf) pdf[i] = df_from_double(v);
  }
}

template <typename TZ>
__global__ void k_cg_newdir(double* __restrict__ p, const TZ* __restrict__ zs, int64_t n, const double* scal,
                            df64* __restrict__ pdf) {
  pdl_entry();
  cg_newdir_body<TZ>(plain_block(), p, zs, n, scal, pdf);
}

// y = x (accumulate = 0) or y += x (accumulate = 1), x double-float, y FP64
__device__ __forceinline__ void join_df64_body(BlockIdx bi_, const df64* __restrict__ x, double* __restrict__ y,
                                               int64_t n, int accumulate) {
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    y[i] = accumulate ? y[i] + df_to_double(x[i]) : df_to_double(x[i]);
}

__global__ void k_join_df64(const df64* __restrict__ x, double* __restrict__ y, int64_t n, int accumulate) {
  pdl_entry();
  join_df64_body(plain_block(), x, y, n, accumulate);
}

__device__ __forceinline__ void split_df64_body(BlockIdx bi_, const double* __restrict__ x, df64* __restrict__ y,
                                                int64_t n) {
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    y[i] = df_from_double(x[i]);
}

__global__ void k_split_df64(const double* __restrict__ x, df64* __restrict__ y, int64_t n) {
  pdl_entry();
  split_df64_body(plain_block(), x, y, n);
}

// q = qdf as FP64 and the partial sums of p . q
__device__ __forceinline__ void dot_dfq_body(BlockIdx bi_, const double* __restrict__ p, const df64* __restrict__ qdf,
                                             double* __restrict__ q, int64_t n, double* partial) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x) {
    const double qi = df_to_double(qdf[i]);
    q[i] = qi;
    acc += p[i] * qi;
  }
  const double b = block_reduce(acc, sh);
  if (threadIdx.x == 0) partial[bi_.b] = b;
}

__global__ void __launch_bounds__(kThreads) k_dot_dfq(const double* __restrict__ p, const df64* __restrict__ qdf,
                                  double* __restrict__ q, int64_t n, double* partial) {
  pdl_entry();
  dot_dfq_body(plain_block(), p, qdf, q, n, partial);
}

__device__ __forceinline__ void add_body(BlockIdx bi_, double* __restrict__ y, const double* __restrict__ x,
                                         int64_t n) {
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    y[i] += x[i];
}

__global__ void k_add(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  pdl_entry();
  add_body(plain_block(), y, x, n);
}

__device__ __forceinline__ void to_f32_body(BlockIdx bi_, const double* __restrict__ x, float* __restrict__ y,
                                            int64_t n, const double* scal, int slot) {
  __shared__ double s_s;
  if (threadIdx.x == 0) {
    double v = 1.0;
    if (slot >= 0) {
      const double nrm = sqrt(scal[slot]);
      v = nrm > 0.0 ? 1.0 / nrm : 1.0;
    }
    s_s = v;
  }
  __syncthreads();
  const double s = s_s;
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    y[i] = (float)(x[i] * s);
}

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n, const double* scal, int slot) {
  pdl_entry();
  to_f32_body(plain_block(), x, y, n, scal, slot);
}

__device__ __forceinline__ void from_f32_body(BlockIdx bi_, const float* __restrict__ x, double* __restrict__ y,
                                              int64_t n, const double* scal, int slot) {
  __shared__ double s_s;
  if (threadIdx.x == 0) {
    double v = 1.0;
    if (slot >= 0) {
      const double nrm = sqrt(scal[slot]);
      v = nrm > 0.0 ? nrm : 1.0;
    }
    s_s = v;
  }
  __syncthreads();
  const double s = s_s;
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    y[i] = (double)x[i] * s;
}

__global__ void k_from_f32(const float* __restrict__ x, double* __restrict__ y, int64_t n, const double* scal,
                           int slot) {
  pdl_entry();
  from_f32_body(plain_block(), x, y, n, scal, slot);
}

struct MassArgs {
  const double* tab;
  int64_t mass[3];
  int n;
  int64_t Ne;
};

__device__ __forceinline__ double mass_at(const MassArgs& a, int64_t dof) {
  const int n = a.n, n3 = n * n * n;
  const int loc = (int)(dof % n3);
  const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
  return a.tab[a.mass[0] + i] * a.tab[a.mass[1] + j] * a.tab[a.mass[2] + k];
}

// partial sums of M f (slot 0) and M (slot 1)
__global__ void __launch_bounds__(kThreads) k_mass_partial(MassArgs a, const double* __restrict__ f, double* partial) {
  pdl_entry();
  __shared__ double sh[kThreads];
  const int64_t total = a.Ne * a.n * a.n * a.n;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double m = mass_at(a, i);
    s0 += m * f[i];
    s1 += m;
  }
  double r0 = block_reduce(s0, sh);
  __syncthreads();
  double r1 = block_reduce(s1, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = r0;
    partial[gridDim.x + blockIdx.x] = r1;
  }
}

__global__ void k_rhs(MassArgs a, const double* __restrict__ f, double* __restrict__ b, const double* scal) {
  pdl_entry();
  const double fbar = scal[kSlotMassF] / scal[kSlotMass];
  const int64_t total = a.Ne * a.n * a.n * a.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = mass_at(a, i) * (f[i] - fbar);
}

__global__ void k_coords(const double* tab, int64_t nodes, int n, int64_t Ne, int nx, int ny, double hx, double hy,
                         double hz, double* x, double* y, double* z) {
  pdl_entry();
  const int n3 = n * n * n;
  const int64_t total = Ne * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / n3;
    const int loc = (int)(idx - e * n3);
    const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    x[idx] = ex * hx + (tab[nodes + i] + 1.0) * 0.5 * hx;
    y[idx] = ey * hy + (tab[nodes + j] + 1.0) * 0.5 * hy;
    z[idx] = ez * hz + (tab[nodes + k] + 1.0) * 0.5 * hz;
  }
}

template <typename T>
__device__ __forceinline__ void zero_body(BlockIdx bi_, T* x, int64_t n) {
  for (int64_t i = bi_.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi_.g * blockDim.x)
    x[i] = (T)0;
}

template <typename T>
__global__ void k_zero(T* x, int64_t n) {
  pdl_entry();
  zero_body<T>(plain_block(), x, n);
}

// Blocks of the two-stage reductions: about 1024 elements per block, at most
// kRedBlocks (8 per SM; vectors above 1.2 M elements); the second stage sums
// the partials of exactly these blocks, so the order of summation is a fixed
// function of n.
inline int red_blocks(int64_t n) {
  const int64_t b = (n + 1023) / 1024;
  return (int)(b < 1 ? 1 : (b > kRedBlocks ? kRedBlocks : b));
}

inline int grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
cudaError_t reduce(const mg_ctx* c, const T* x, const T* y, int64_t n, int mode, int slot) {
  const int nb = red_blocks(n);
  launch_pdl<partial_body<T>>(k_partial<T>, nb, kThreads, 0, c->stream, x, y, n, mode, c->ws.red);
  c->nlaunch += 1;
  launch_pdl<final_body>(k_final, 1, kThreads, 0, c->stream, c->ws.red, nb, c->ws.scal, slot);
  c->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace

int reduction_blocks(int64_t n) { return red_blocks(n); }

cudaError_t launch_final_sum(const mg_ctx* c, int nb, int slot) {
  launch_pdl<final_body>(k_final, 1, kThreads, 0, c->stream, c->ws.red, nb, c->ws.scal, slot);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_update_final(const mg_ctx* c, int nb, int64_t n) {
  launch_pdl<cg_update_final_body>(k_cg_update_final, 1, kThreads, 0, c->stream, c->ws.red, nb, c->ws.scal, n);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_dot(const mg_ctx* c, const double* x, const double* y, int64_t n, int slot) {
  return reduce<double>(c, x, y, n, 0, slot);
}

cudaError_t launch_sum(const mg_ctx* c, const double* x, int64_t n, int slot) {
  return reduce<double>(c, x, x, n, 1, slot);
}

cudaError_t launch_sub_mean(const mg_ctx* c, double* x, int64_t n, int sum_slot) {
  launch_pdl<sub_mean_body<double>>(k_sub_mean<double>, grid_for(n), kThreads, 0, c->stream, x, n, c->ws.scal,
                                    sum_slot);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_cg_update(const mg_ctx* c, double* x, const double* p, double* r, const double* q, int64_t n) {
  const int nb = red_blocks(n);
  launch_pdl<cg_update_body>(k_cg_update, nb, kThreads, 0, c->stream, x, p, r, q, n, c->ws.scal, c->ws.red);
  launch_pdl<cg_update_final_body>(k_cg_update_final, 1, kThreads, 0, c->stream, c->ws.red, nb, c->ws.scal, n);
  c->nlaunch += 2;
  return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_cg_direction(const mg_ctx* c, double* p, const TZ* z, const double* q, const double* r, int64_t n,
                                df64* pdf) {
  const int nb = red_blocks(n);
  launch_pdl<cg_sums_body<TZ>>(k_cg_sums<TZ>, nb, kThreads, 0, c->stream, z, q, r, n, c->ws.red);
  launch_pdl<cg_sums_final_body<TZ>>(k_cg_sums_final<TZ>, 1, kThreads, 0, c->stream, c->ws.red, nb, c->ws.scal, n);
  launch_pdl<cg_newdir_body<TZ>>(k_cg_newdir<TZ>, grid_for(n), kThreads, 0, c->stream, p, z, n, c->ws.scal, pdf);
  c->nlaunch += 3;
  return cudaGetLastError();
}

template cudaError_t launch_cg_direction<double>(const mg_ctx*, double*, const double*, const double*,
                                                 const double*, int64_t, df64*);
template cudaError_t launch_cg_direction<float>(const mg_ctx*, double*, const float*, const double*, const double*,
                                                int64_t, df64*);
template cudaError_t launch_cg_direction<df64>(const mg_ctx*, double*, const df64*, const double*, const double*,
                                               int64_t, df64*);

cudaError_t launch_split_df64(const mg_ctx* c, const double* x, df64* y, int64_t n) {
  launch_pdl<split_df64_body>(k_split_df64, grid_for(n), kThreads, 0, c->stream, x, y, n);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_join_df64(const mg_ctx* c, const df64* x, double* y, int64_t n, int accumulate) {
  launch_pdl<join_df64_body>(k_join_df64, grid_for(n), kThreads, 0, c->stream, x, y, n, accumulate);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_dot_dfq(const mg_ctx* c, const double* p, const df64* qdf, double* q, int64_t n, int slot) {
  const int nb = red_blocks(n);
  launch_pdl<dot_dfq_body>(k_dot_dfq, nb, kThreads, 0, c->stream, p, qdf, q, n, c->ws.red);
  launch_pdl<final_body>(k_final, 1, kThreads, 0, c->stream, c->ws.red, nb, c->ws.scal, slot);
  c->nlaunch += 2;
  return cudaGetLastError();
}

cudaError_t launch_add(const mg_ctx* c, double* y, const double* x, int64_t n) {
  launch_pdl<add_body>(k_add, grid_for(n), kThreads, 0, c->stream, y, x, n);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const mg_ctx* c, const double* x, float* y, int64_t n, int norm_slot) {
  launch_pdl<to_f32_body>(k_to_f32, grid_for(n), kThreads, 0, c->stream, x, y, n, c->ws.scal, norm_slot);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_from_f32(const mg_ctx* c, const float* x, double* y, int64_t n, int norm_slot) {
  launch_pdl<from_f32_body>(k_from_f32, grid_for(n), kThreads, 0, c->stream, x, y, n, c->ws.scal, norm_slot);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_rhs(const mg_ctx* c, const double* f, double* b) {
  if (c->graded) return launch_grhs(c, f, b);
  const LevelInfo& lv = c->lev[c->L];
  MassArgs a;
  a.tab = c->ws.tab64;
  for (int d = 0; d < 3; ++d) a.mass[d] = lv.t[d].mass;
  a.n = lv.n;
  a.Ne = c->Ne;
  const int nb = red_blocks(lv.N);
  launch_pdl(k_mass_partial, nb, kThreads, 0, c->stream, a, f, c->ws.red);
  c->nlaunch += 1;
  launch_pdl<final_body>(k_final, 1, kThreads, 0, c->stream, c->ws.red, nb, c->ws.scal, kSlotMassF);
  c->nlaunch += 1;
  launch_pdl<final_body>(k_final, 1, kThreads, 0, c->stream, c->ws.red + nb, nb, c->ws.scal, kSlotMass);
  c->nlaunch += 1;
  launch_pdl(k_rhs, grid_for(lv.N), kThreads, 0, c->stream, a, f, b, c->ws.scal);
  c->nlaunch += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_sum(c, b, lv.N, kSlotSum)) != cudaSuccess) return e;
  return launch_sub_mean(c, b, lv.N, kSlotSum);
}

cudaError_t launch_coords(const mg_ctx* c, int l, double* x, double* y, double* z) {
  if (c->graded) return launch_gcoords(c, l, x, y, z);
  const LevelInfo& lv = c->lev[l];
  launch_pdl(k_coords, grid_for(lv.N), kThreads, 0, c->stream, c->ws.tab64, lv.t[0].nodes, lv.n, c->Ne, c->ne[0], c->ne[1],
                                                        lv.h[0], lv.h[1], lv.h[2], x, y, z);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero(const mg_ctx* c, T* x, int64_t n) {
  launch_pdl<zero_body<T>>(k_zero<T>, grid_for(n), kThreads, 0, c->stream, x, n);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template cudaError_t launch_zero<double>(const mg_ctx*, double*, int64_t);
template cudaError_t launch_zero<float>(const mg_ctx*, float*, int64_t);
template cudaError_t launch_zero<df64>(const mg_ctx*, df64*, int64_t);

}  // namespace mgdg
