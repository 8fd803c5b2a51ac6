// Vector kernels of the outer MG-CG iteration in double-float arithmetic
// (mg_opts.outer_df64 = 2; Section 3.2, the inexact preconditioned CG).
//
// On this GPU the FP64 pipe runs at 1/61 of the FP32 rate, and the FP64 CG
// vector passes, with their two to six FP64 operations per element, keep it
// busy (ncu: FP64 pipe 77-85 % in the update, direction and inner-product
// passes of the mixed solve).  Here the outer vectors x, r, p, q are stored as
// double-float pairs (df64.cuh, about 48 significant bits) and every
// per-element operation runs on the FP32 pipes; the per-thread sums are
// compensated double-float sums, and only the per-block totals (a few
// thousand values) are added in FP64, in the fixed two-stage order of the
// FP64 reductions, so repeated runs give identical bits.  The preconditioner
// input is written by the update pass itself (r scaled by the previous
// residual norm, in FP32), and the scale is kept in a device slot for the
// direction pass.
#include "mg_internal.h"

namespace mgdg {
namespace {

constexpr int kT = 256;

// FP64 reduction of a few thousand per-block totals (the second stages).
__device__ double odf_block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Block total of one double-float value per thread, in a fixed order:
// pair additions across each warp (FP32 pipes), then the eight warp totals
// in FP64 by thread 0 (the only thread that receives the total).  Keeping
// the per-element and per-thread work off the FP64 pipe is the point: ncu
// counted a per-thread FP64 tree at 40 % of the FP64 pipe in these passes.
__device__ double odf_block_total(df64 v, df64* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df64 w(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    v = v + w;
  }
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (double)sh[w].hi + (double)sh[w].lo;
  __syncthreads();
  return t;
}

__device__ __forceinline__ Acc<df64> odf_zero() {
  Acc<df64> a;
  a.s = 0.f;
  a.c = 0.f;
  return a;
}


// partial[b] = sum p . q over block b's elements
__device__ __forceinline__ void odf_dot_body(BlockIdx bi, const df64* __restrict__ p, const df64* __restrict__ q,
                                             int64_t n, double* partial) {
  __shared__ df64 sh[kT / 32];
  Acc<df64> acc = odf_zero();
  for (int64_t i = bi.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi.g * blockDim.x)
    acc.add(p[i], q[i]);
  const double b = odf_block_total(acc.get(), sh);
  if (threadIdx.x == 0) partial[bi.b] = b;
}

__global__ void __launch_bounds__(kT) k_odf_dot(const df64* __restrict__ p, const df64* __restrict__ q, int64_t n,
                                                double* partial) {
  pdl_entry();
  odf_dot_body(plain_block(), p, q, n, partial);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; partial sums of r and r.r
// (columns 0, 1); r32 = r / sqrt(rr_old) for the FP32 preconditioner, and
// scal[Scale] = sqrt(rr_old) (the factor that brings its output back).
__device__ __forceinline__ void odf_update_body(BlockIdx bi, df64* __restrict__ x, const df64* __restrict__ p,
                                                df64* __restrict__ r, const df64* __restrict__ q, int64_t n,
                                                double* scal, double* partial, float* __restrict__ r32) {
  __shared__ df64 sh[kT / 32];
  __shared__ df64 s_a;
  __shared__ float s_sc;
  if (threadIdx.x == 0) {  // the scalars once per block
    const double alpha = scal[kSlotRZ] / scal[kSlotPQ];
    const double nrm = sqrt(scal[kSlotRR]);
    s_a = df64(alpha);
    s_sc = nrm > 0.0 ? (float)(1.0 / nrm) : 1.f;
    if (bi.b == 0) {
      scal[kSlotAlpha] = alpha;
      scal[kSlotScale] = nrm > 0.0 ? nrm : 1.0;
    }
  }
  __syncthreads();
  const df64 a = s_a, na = -s_a;
  const float sc = s_sc;
  Acc<df64> s1 = odf_zero(), s2 = odf_zero();
  for (int64_t i = bi.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi.g * blockDim.x) {
    x[i] = x[i] + a * p[i];
    const df64 ri = r[i] + na * q[i];
    r[i] = ri;
    s1.add(ri);
    s2.add(ri, ri);
    r32[i] = __fmul_rn(__fadd_rn(ri.hi, ri.lo), sc);
  }
  const double b1 = odf_block_total(s1.get(), sh);
  const double b2 = odf_block_total(s2.get(), sh);
  if (threadIdx.x == 0) {
    partial[bi.b] = b1;
    partial[bi.g + bi.b] = b2;
  }
}

__global__ void __launch_bounds__(kT) k_odf_update(df64* __restrict__ x, const df64* __restrict__ p,
                                                   df64* __restrict__ r, const df64* __restrict__ q, int64_t n,
                                                   double* scal, double* partial, float* __restrict__ r32) {
  pdl_entry();
  odf_update_body(plain_block(), x, p, r, q, n, scal, partial, r32);
}

// Partial sums of z, z.q, z.r (columns 0 .. 2) of the unscaled FP32 z.
__device__ __forceinline__ void odf_sums_body(BlockIdx bi, const float* __restrict__ z, const df64* __restrict__ q,
                                              const df64* __restrict__ r, int64_t n, double* partial) {
  __shared__ df64 sh[kT / 32];
  Acc<df64> a0 = odf_zero(), a1 = odf_zero(), a2 = odf_zero();
  for (int64_t i = bi.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi.g * blockDim.x) {
    const df64 zi(z[i], 0.f);
    a0.add(zi);
    a1.add(zi, q[i]);
    a2.add(zi, r[i]);
  }
  const double b0 = odf_block_total(a0.get(), sh);
  const double b1 = odf_block_total(a1.get(), sh);
  const double b2 = odf_block_total(a2.get(), sh);
  if (threadIdx.x == 0) {
    partial[bi.b] = b0;
    partial[bi.g + bi.b] = b1;
    partial[2 * bi.g + bi.b] = b2;
  }
}

__global__ void __launch_bounds__(kT) k_odf_sums(const float* __restrict__ z, const df64* __restrict__ q,
                                                 const df64* __restrict__ r, int64_t n, double* partial) {
  pdl_entry();
  odf_sums_body(plain_block(), z, q, r, n, partial);
}

// The three column totals (fixed order) -> with z' = s z - mean(s z) (s =
// scal[Scale]): z'.q = s z.q (1^T q = 0), z'.r' = s z.r - sum(s z) sum(r) / n;
// beta = -alpha z'.q / rz_old (0 for the first direction); rz = z'.r'.
__device__ __forceinline__ void odf_sums_final_body(BlockIdx bi, const double* partial, int nb, double* scal,
                                                    int64_t n, int first) {
  __shared__ double sh[kT];
  double v[3];
  for (int k = 0; k < 3; ++k) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[k * nb + i];
    v[k] = odf_block_sum(acc, sh);
  }
  if (threadIdx.x == 0) {
    const double zsc = scal[kSlotScale], inv = 1.0 / (double)n;
    const double sz = zsc * v[0], zq = zsc * v[1];
    const double zr = zsc * v[2] - sz * scal[kSlotSum] * inv;
    scal[kSlotZQ] = zq;
    scal[kSlotBeta] = first ? 0.0 : -scal[kSlotAlpha] * zq / scal[kSlotRZ];
    scal[kSlotMuZ] = sz * inv;
    scal[kSlotRZ] = zr;
  }
}

__global__ void __launch_bounds__(kT) k_odf_sums_final(const double* partial, int nb, double* scal, int64_t n,
                                                       int first) {
  pdl_entry();
  odf_sums_final_body(plain_block(), partial, nb, scal, n, first);
}

// p = (s z - mu_z) + beta p (first: p = s z - mu_z), double-float
__device__ __forceinline__ void odf_newdir_body(BlockIdx bi, df64* __restrict__ p, const float* __restrict__ z,
                                                int64_t n, const double* scal, int first) {
  __shared__ df64 s_v[3];
  if (threadIdx.x == 0) {  // the scalars once per block
    s_v[0] = df64(scal[kSlotScale]);
    s_v[1] = df64(-scal[kSlotMuZ]);
    s_v[2] = df64(scal[kSlotBeta]);
  }
  __syncthreads();
  const df64 zsc = s_v[0], muz = s_v[1], beta = s_v[2];
  for (int64_t i = bi.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi.g * blockDim.x) {
    const df64 v = df64(z[i], 0.f) * zsc + muz;
    p[i] = first ? v : v + beta * p[i];
  }
}

__global__ void __launch_bounds__(kT) k_odf_newdir(df64* __restrict__ p, const float* __restrict__ z, int64_t n,
                                                   const double* scal, int first) {
  pdl_entry();
  odf_newdir_body(plain_block(), p, z, n, scal, first);
}

// Partial sums of r and r.r (columns 0, 1) of a double-float vector.
__device__ __forceinline__ void odf_rsums_body(BlockIdx bi, const df64* __restrict__ r, int64_t n, double* partial) {
  __shared__ df64 sh[kT / 32];
  Acc<df64> s1 = odf_zero(), s2 = odf_zero();
  for (int64_t i = bi.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi.g * blockDim.x) {
    const df64 ri = r[i];
    s1.add(ri);
    s2.add(ri, ri);
  }
  const double b1 = odf_block_total(s1.get(), sh);
  const double b2 = odf_block_total(s2.get(), sh);
  if (threadIdx.x == 0) {
    partial[bi.b] = b1;
    partial[bi.g + bi.b] = b2;
  }
}

__global__ void __launch_bounds__(kT) k_odf_rsums(const df64* __restrict__ r, int64_t n, double* partial) {
  pdl_entry();
  odf_rsums_body(plain_block(), r, n, partial);
}

// FP64 -> double-float in place (the same 8 bytes per value); FP64 pipe, once per solve
__device__ __forceinline__ void odf_split_body(BlockIdx bi, double* v, int64_t n) {
  for (int64_t i = bi.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi.g * blockDim.x) {
    const double d = v[i];
    reinterpret_cast<df64*>(v)[i] = df_from_double(d);
  }
}

__global__ void __launch_bounds__(kT) k_odf_split(double* v, int64_t n) {
  pdl_entry();
  odf_split_body(plain_block(), v, n);
}

// y = r / sqrt(rr) in FP32 and scal[Scale] = sqrt(rr): the first preconditioner input
__device__ __forceinline__ void odf_to_f32_body(BlockIdx bi, const df64* __restrict__ r, float* __restrict__ y,
                                                int64_t n, double* scal) {
  __shared__ float s_sc;
  if (threadIdx.x == 0) {  // the scale once per block
    const double nrm = sqrt(scal[kSlotRR]);
    s_sc = nrm > 0.0 ? (float)(1.0 / nrm) : 1.f;
    if (bi.b == 0) scal[kSlotScale] = nrm > 0.0 ? nrm : 1.0;
  }
  __syncthreads();
  const float sc = s_sc;
  for (int64_t i = bi.b * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)bi.g * blockDim.x)
    y[i] = __fmul_rn(__fadd_rn(r[i].hi, r[i].lo), sc);
}

__global__ void __launch_bounds__(kT) k_odf_to_f32(const df64* __restrict__ r, float* __restrict__ y, int64_t n,
                                                   double* scal) {
  pdl_entry();
  odf_to_f32_body(plain_block(), r, y, n, scal);
}

inline int odf_grid(int64_t n) {
  int64_t b = (n + kT - 1) / kT;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_odf_update(const mg_ctx* c, df64* x, const df64* p, df64* r, const df64* q, float* r32,
                              int64_t n) {
  cudaError_t e;
  const int nb = reduction_blocks(n);
  launch_pdl<odf_dot_body>(k_odf_dot, nb, kT, 0, c->stream, p, q, n, c->ws.red);
  c->nlaunch += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_final_sum(c, nb, kSlotPQ)) != cudaSuccess) return e;
  launch_pdl<odf_update_body>(k_odf_update, nb, kT, 0, c->stream, x, p, r, q, n, c->ws.scal, c->ws.red, r32);
  c->nlaunch += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_update_final(c, nb, n);
}

cudaError_t launch_odf_direction(const mg_ctx* c, df64* p, const float* z, const df64* q, const df64* r, int64_t n,
                                 int first) {
  const int nb = reduction_blocks(n);
  launch_pdl<odf_sums_body>(k_odf_sums, nb, kT, 0, c->stream, z, q, r, n, c->ws.red);
  launch_pdl<odf_sums_final_body>(k_odf_sums_final, 1, kT, 0, c->stream, c->ws.red, nb, c->ws.scal, n, first);
  launch_pdl<odf_newdir_body>(k_odf_newdir, odf_grid(n), kT, 0, c->stream, p, z, n, c->ws.scal, first);
  c->nlaunch += 3;
  return cudaGetLastError();
}

cudaError_t launch_odf_residual_norm(const mg_ctx* c, const df64* r, int64_t n) {
  const int nb = reduction_blocks(n);
  launch_pdl<odf_rsums_body>(k_odf_rsums, nb, kT, 0, c->stream, r, n, c->ws.red);
  c->nlaunch += 1;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_update_final(c, nb, n);
}

cudaError_t launch_odf_split(const mg_ctx* c, double* v, int64_t n) {
  launch_pdl<odf_split_body>(k_odf_split, odf_grid(n), kT, 0, c->stream, v, n);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_odf_to_f32(const mg_ctx* c, const df64* r, float* y, int64_t n) {
  launch_pdl<odf_to_f32_body>(k_odf_to_f32, odf_grid(n), kT, 0, c->stream, r, y, n, c->ws.scal);
  c->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace mgdg
