// FP32 fast-diagonalisation smoother with the 1D factors in the kernel's
// parameter space (Section 3.1, the subdomain solve
//   du_s = (Sz(x)Sy(x)Sx) (Lx (+) Ly (+) Lz)^{-1} (Sz^T(x)Sy^T(x)Sx^T) r_s).
//
// In FP32 the line products of the shared-memory kernel (fdm_tmpl.cuh) are
// limited by their loads, not by the FMA pipe: every multiply-add reads its
// coefficient of S from shared memory.  Here the even/odd halves of the six
// 1D factors (at most 29.4 KB at m = 35) travel as one __grid_constant__
// kernel parameter, so with the fully unrolled products of a compile-time
// width every coefficient is an immediate constant-bank operand of its FMA:
// the only shared-memory traffic left is the subdomain tile itself.
//
// One block takes SPB subdomains, one thread per 1D line and pass: the first
// pass gathers the x-lines of r_s = R_s r from the element and its
// neighbours and transforms them into the shared-memory tile, three more run
// in place (y forward; z forward, division by the eigenvalue sums, z
// backward; y backward), and the last (x backward, weights folded into SW)
// writes the weighted correction tile to the correction buffer, in the layout
// of the other smoother kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cmath>

#include <algorithm>
#include <atomic>

#include "mg_internal.h"

namespace mgdg {
namespace {

template <int M>
struct FdmCShape {
  static constexpr int h = M / 2, ne = h + 1, ho = h > 0 ? h : 1;
  static constexpr int M2 = M * M, M3 = M2 * M;
  static constexpr int spb = M2 >= 256 ? 1 : 256 / M2;     // subdomains per block
  static constexpr int lines = spb * M2;                     // lines of one pass
  static constexpr int iters = (lines + 511) / 512;
  static constexpr int threads = ((lines + iters - 1) / iters + 31) / 32 * 32;
  static constexpr size_t smem = sizeof(float) * (size_t)spb * M3;
};

template <int M>
struct FdmCArgs {
  using Sh = FdmCShape<M>;
  const float* r;
  float* corr;
  const float* dinv;                 // 1 / (lam_x[i] + lam_y[j] + lam_z[k]) at i + M (j + M k)
  int64_t Ne;
  int nx, ny, nz, n, no;
  float se[3][Sh::ne * Sh::ne];      // S[a][p], a, p <= h         (forward, even modes)
  float so[3][Sh::ho * Sh::ho];      // S[a][h+1+q], a, q < h      (forward, odd modes)
  float we[3][Sh::ne * Sh::ne];      // SW[a][p], a, p <= h        (backward, even modes)
  float wo[3][Sh::ho * Sh::ho];      // SW[a][h+1+q], a, q < h     (backward, odd modes)
};

// y = S_d^T x (even modes first), x a reflection-symmetric line.
template <int M, int D>
__device__ __forceinline__ void fwd_c(const FdmCArgs<M>& a, const float (&x)[M], float (&y)[M]) {
  constexpr int h = M / 2, ne = h + 1;
  float e[ne], o[h > 0 ? h : 1];
#pragma unroll
  for (int t = 0; t < h; ++t) {
    e[t] = x[t] + x[M - 1 - t];
    o[t] = x[t] - x[M - 1 - t];
  }
  e[h] = x[h];
#pragma unroll
  for (int p = 0; p < ne; ++p) {
    float acc = a.se[D][p] * e[0];
#pragma unroll
    for (int t = 1; t < ne; ++t) acc = fmaf(a.se[D][t * ne + p], e[t], acc);
    y[p] = acc;
  }
#pragma unroll
  for (int q = 0; q < h; ++q) {
    float acc = a.so[D][q] * o[0];
#pragma unroll
    for (int t = 1; t < h; ++t) acc = fmaf(a.so[D][t * h + q], o[t], acc);
    y[ne + q] = acc;
  }
}

// x = SW_d v (weights folded into SW).
template <int M, int D>
__device__ __forceinline__ void bwd_c(const FdmCArgs<M>& a, const float (&v)[M], float (&x)[M]) {
  constexpr int h = M / 2, ne = h + 1;
#pragma unroll
  for (int t = 0; t <= h; ++t) {
    float E = a.we[D][t * ne] * v[0];
#pragma unroll
    for (int p = 1; p < ne; ++p) E = fmaf(a.we[D][t * ne + p], v[p], E);
    if (t < h) {
      float O = a.wo[D][t * h] * v[ne];
#pragma unroll
      for (int q = 1; q < h; ++q) O = fmaf(a.wo[D][t * h + q], v[ne + q], O);
      x[t] = E + O;
      x[M - 1 - t] = E - O;
    } else {
      x[t] = E;
    }
  }
}

__device__ __forceinline__ int fc_wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// Operand emulation for a precision study (mg_opts.fdm_operands): every
// line entering a 1D product is rounded (OP = 1: to BF16, nearest even;
// OP = 2: to FP8 E4M3, nearest even, after scaling the line by the power of
// two that puts its largest magnitude in [224, 448)) and the 1D factors were
// rounded the same way on the host (FP8: per output index), the products
// accumulating in FP32 -- the arithmetic of BF16 / FP8 tensor-core
// contractions with FP32 accumulation and scaled eigenbases, on the CUDA cores.
template <int OP, int M>
__device__ __forceinline__ void round_line(float (&x)[M]) {
  if constexpr (OP == 1) {
#pragma unroll
    for (int t = 0; t < M; ++t) x[t] = __bfloat162float(__float2bfloat16_rn(x[t]));
  } else if constexpr (OP == 2) {
    float amax = 0.f;
#pragma unroll
    for (int t = 0; t < M; ++t) amax = fmaxf(amax, fabsf(x[t]));
    if (amax > 0.f) {
      int e;
      frexpf(amax / 448.f, &e);  // amax / 448 = f 2^e, f in [0.5, 1)
      const float sc = ldexpf(1.f, e), inv = ldexpf(1.f, -e);
#pragma unroll
      for (int t = 0; t < M; ++t) {
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(x[t] * inv, __NV_SATFINITE, __NV_E4M3);
        x[t] = __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))) * sc;
      }
    }
  }
}

template <int M, int OP>
__global__ void __launch_bounds__(FdmCShape<M>::threads) k_fdm_c(const __grid_constant__ FdmCArgs<M> a) {
  pdl_entry();
  using Sh = FdmCShape<M>;
  constexpr int M2 = Sh::M2, M3 = Sh::M3, SPB = Sh::spb;
  extern __shared__ __align__(16) float fc_tile[];  // SPB tiles of M^3, node (i, j, k) at i + M (j + M k)
  const int n = a.n, no = a.no, n3 = n * n * n;
  const float* __restrict__ dinv = a.dinv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t s0 = (int64_t)blockIdx.x * SPB; s0 < a.Ne; s0 += (int64_t)gridDim.x * SPB) {
    const int lines = (int)(a.Ne - s0 < SPB ? a.Ne - s0 : SPB) * M2;
    // pass 1: gather the x-lines of r_s = R_s r (left strip, element, right
    // strip), x forward
    for (int ln = tid; ln < lines; ln += nt) {
      const int g = ln / M2, l2 = ln - g * M2, b = l2 % M, c = l2 / M;
      const int s = (int)(s0 + g), sxy = s / a.nx;  // element indices fit in 32 bits
      const int sx = s - sxy * a.nx, sy = sxy % a.ny, sz = sxy / a.ny;
      const int dy = b < no ? -1 : (b < no + n ? 0 : 1), iy = b - no + (dy < 0 ? n : (dy > 0 ? -n : 0));
      const int dz = c < no ? -1 : (c < no + n ? 0 : 1), iz = c - no + (dz < 0 ? n : (dz > 0 ? -n : 0));
      const int64_t row = (int64_t)a.nx * (fc_wrap(sy + dy, a.ny) + (int64_t)a.ny * fc_wrap(sz + dz, a.nz));
      const int loc = n * (iy + n * iz);
      // position t of the line in the left / centre / right element
      const float* rl = a.r + (fc_wrap(sx - 1, a.nx) + row) * n3 + loc + (n - no);
      const float* rc = a.r + (sx + row) * n3 + loc - no;
      const float* rr = a.r + (fc_wrap(sx + 1, a.nx) + row) * n3 + loc - (no + n);
      float x[M], y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = __ldg((t < no ? rl : (t < no + n ? rc : rr)) + t);
      round_line<OP>(x);
      fwd_c<M, 0>(a, x, y);
      float* line = fc_tile + g * M3 + M * l2;
#pragma unroll
      for (int t = 0; t < M; ++t) line[t] = y[t];
    }
    __syncthreads();
    // pass 2: y forward
    for (int ln = tid; ln < lines; ln += nt) {
      const int l2 = ln % M2;
      float* line = fc_tile + (ln / M2) * M3 + (l2 % M) + M2 * (l2 / M);
      float x[M], y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = line[t * M];
      round_line<OP>(x);
      fwd_c<M, 1>(a, x, y);
#pragma unroll
      for (int t = 0; t < M; ++t) line[t * M] = y[t];
    }
    __syncthreads();
    // pass 3: z forward, times 1 / (lam_x + lam_y + lam_z), z backward
    for (int ln = tid; ln < lines; ln += nt) {
      const int l2 = ln % M2;
      float* line = fc_tile + (ln / M2) * M3 + l2;
      float x[M], y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = line[t * M2];
      round_line<OP>(x);
      fwd_c<M, 2>(a, x, y);
#pragma unroll
      for (int t = 0; t < M; ++t) y[t] *= __ldg(dinv + l2 + t * M2);
      round_line<OP>(y);
      bwd_c<M, 2>(a, y, x);
#pragma unroll
      for (int t = 0; t < M; ++t) line[t * M2] = x[t];
    }
    __syncthreads();
    // pass 4: y backward
    for (int ln = tid; ln < lines; ln += nt) {
      const int l2 = ln % M2;
      float* line = fc_tile + (ln / M2) * M3 + (l2 % M) + M2 * (l2 / M);
      float x[M], y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) y[t] = line[t * M];
      round_line<OP>(y);
      bwd_c<M, 1>(a, y, x);
#pragma unroll
      for (int t = 0; t < M; ++t) line[t * M] = x[t];
    }
    __syncthreads();
    // pass 5: x backward (weights folded into SW), straight to the correction buffer
    for (int ln = tid; ln < lines; ln += nt) {
      const int g = ln / M2, l2 = ln - g * M2;
      const float* line = fc_tile + g * M3 + M * l2;
      float* out = a.corr + (s0 + g) * M3 + M * l2;
      float x[M], y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) y[t] = line[t];
      round_line<OP>(y);
      bwd_c<M, 0>(a, y, x);
#pragma unroll
      for (int t = 0; t < M; ++t) out[t] = x[t];
    }
    __syncthreads();
  }
}

// ---- the same solve split into three grid-wide kernels ----
//
// The passes are independent across planes of the tile, so they can be
// spread over three kernels with many blocks each, the tile staying in the
// correction buffer between them: a level with few subdomains (the 4^3 mesh
// at P = 32 has 64) then fills the 152 SMs, and on every cubic level from
// m = 11 up it was measured faster than the one-kernel form (the default
// there):
//   k_fdm_xy: per block SL z-planes (c) of one subdomain: gather the x-lines,
//             x forward, y forward;
//   k_fdm_z:  one thread per (i, j) column of every subdomain: z forward,
//             times 1 / (lam_x + lam_y + lam_z), z backward, in place;
//   k_fdm_yx: per block SL z-planes: y backward, x backward (weights folded
//             into SW), the weighted correction written back in place.
// Every line sees exactly the products of k_fdm_c, in the same order.  (FP32
// operands only: the operand studies run the one-kernel form.)
template <int M>
struct FdmSplitShape {
  static constexpr int M2 = M * M, M3 = M2 * M;
  static constexpr int sl = 160 / M < 1 ? 1 : 160 / M;  // planes per block: about 160 threads
  static constexpr int sl_c = sl < M ? sl : M;
  static constexpr int threads = (sl_c * M + 31) / 32 * 32;
  static constexpr int groups = (M + sl_c - 1) / sl_c;        // plane groups per subdomain
  static constexpr int zt = 256;                               // columns per block of k_fdm_z
  static constexpr size_t smem = sizeof(float) * (size_t)sl_c * M2;
};

template <int M>
__global__ void __launch_bounds__(FdmSplitShape<M>::threads) k_fdm_xy(const __grid_constant__ FdmCArgs<M> a) {
  pdl_entry();
  using Sh = FdmSplitShape<M>;
  constexpr int M2 = Sh::M2, SL = Sh::sl_c;
  extern __shared__ __align__(16) float fs_tile[];  // SL planes, node (p, b) of plane g at g M^2 + p + M b
  const int n = a.n, no = a.no, n3 = n * n * n;
  const int64_t s = blockIdx.x / Sh::groups;
  const int c0 = (int)(blockIdx.x - s * Sh::groups) * SL;
  const int planes = M - c0 < SL ? M - c0 : SL;
  const int tid = threadIdx.x;
  if (s >= a.Ne) return;
  const int sxy = (int)s / a.nx;
  const int sx = (int)s - sxy * a.nx, sy = sxy % a.ny, sz = sxy / a.ny;
  // x-lines (b, c): gather and x forward
  if (tid < planes * M) {
    const int g = tid / M, b = tid - g * M, c = c0 + g;
    const int dy = b < no ? -1 : (b < no + n ? 0 : 1), iy = b - no + (dy < 0 ? n : (dy > 0 ? -n : 0));
    const int dz = c < no ? -1 : (c < no + n ? 0 : 1), iz = c - no + (dz < 0 ? n : (dz > 0 ? -n : 0));
    const int64_t row = (int64_t)a.nx * (fc_wrap(sy + dy, a.ny) + (int64_t)a.ny * fc_wrap(sz + dz, a.nz));
    const int loc = n * (iy + n * iz);
    const float* rl = a.r + (fc_wrap(sx - 1, a.nx) + row) * n3 + loc + (n - no);
    const float* rc = a.r + (sx + row) * n3 + loc - no;
    const float* rr = a.r + (fc_wrap(sx + 1, a.nx) + row) * n3 + loc - (no + n);
    float x[M], y[M];
#pragma unroll
    for (int t = 0; t < M; ++t) x[t] = __ldg((t < no ? rl : (t < no + n ? rc : rr)) + t);
    fwd_c<M, 0>(a, x, y);
    float* line = fs_tile + g * M2 + M * b;
#pragma unroll
    for (int t = 0; t < M; ++t) line[t] = y[t];
  }
  __syncthreads();
  // y-lines (p, c): y forward, to plane c of the tile in the correction buffer
  if (tid < planes * M) {
    const int g = tid / M, p = tid - g * M;
    const float* line = fs_tile + g * M2 + p;
    float* out = a.corr + s * Sh::M3 + (int64_t)(c0 + g) * M2 + p;
    float x[M], y[M];
#pragma unroll
    for (int t = 0; t < M; ++t) x[t] = line[t * M];
    fwd_c<M, 1>(a, x, y);
#pragma unroll
    for (int t = 0; t < M; ++t) out[t * M] = y[t];
  }
}

template <int M>
__global__ void __launch_bounds__(FdmSplitShape<M>::zt) k_fdm_z(const __grid_constant__ FdmCArgs<M> a) {
  pdl_entry();
  using Sh = FdmSplitShape<M>;
  constexpr int M2 = Sh::M2;
  const int64_t col = (int64_t)blockIdx.x * Sh::zt + threadIdx.x;
  const int64_t s = col / M2;
  const int l2 = (int)(col - s * M2);
  if (s >= a.Ne) return;
  float* line = a.corr + s * Sh::M3 + l2;
  float x[M], y[M];
#pragma unroll
  for (int t = 0; t < M; ++t) x[t] = line[(int64_t)t * M2];
  fwd_c<M, 2>(a, x, y);
#pragma unroll
  for (int t = 0; t < M; ++t) y[t] *= __ldg(a.dinv + l2 + t * M2);
  bwd_c<M, 2>(a, y, x);
#pragma unroll
  for (int t = 0; t < M; ++t) line[(int64_t)t * M2] = x[t];
}

template <int M>
__global__ void __launch_bounds__(FdmSplitShape<M>::threads) k_fdm_yx(const __grid_constant__ FdmCArgs<M> a) {
  pdl_entry();
  using Sh = FdmSplitShape<M>;
  constexpr int M2 = Sh::M2, SL = Sh::sl_c;
  extern __shared__ __align__(16) float fs_tile[];
  const int64_t s = blockIdx.x / Sh::groups;
  const int c0 = (int)(blockIdx.x - s * Sh::groups) * SL;
  const int planes = M - c0 < SL ? M - c0 : SL;
  const int tid = threadIdx.x;
  if (s >= a.Ne) return;
  float* plane0 = a.corr + s * Sh::M3 + (int64_t)c0 * M2;
  // y-lines (p, c): y backward into shared memory
  if (tid < planes * M) {
    const int g = tid / M, p = tid - g * M;
    const float* in = plane0 + g * M2 + p;
    float* line = fs_tile + g * M2 + p;
    float x[M], y[M];
#pragma unroll
    for (int t = 0; t < M; ++t) y[t] = in[t * M];
    bwd_c<M, 1>(a, y, x);
#pragma unroll
    for (int t = 0; t < M; ++t) line[t * M] = x[t];
  }
  __syncthreads();
  // x-lines (b, c): x backward, in place in shared memory
  if (tid < planes * M) {
    const int g = tid / M, b = tid - g * M;
    float* line = fs_tile + g * M2 + M * b;
    float x[M], y[M];
#pragma unroll
    for (int t = 0; t < M; ++t) y[t] = line[t];
    bwd_c<M, 0>(a, y, x);
#pragma unroll
    for (int t = 0; t < M; ++t) line[t] = x[t];
  }
  __syncthreads();
  // the planes are contiguous in the correction tile: coalesced copy out
  for (int i = tid; i < planes * M2; i += blockDim.x) plane0[i] = fs_tile[i];
}

// Host-side fill of the parameter block from the FP32 tables of level l.
inline float round_bf16_host(float v) {
  // nearest BF16 (ties to even) of a finite FP32 value
  uint32_t u;
  memcpy(&u, &v, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  memcpy(&v, &u, 4);
  return v;
}

// Nearest FP8 E4M3 value of a finite v (1 sign bit, 4 exponent bits with
// bias 7, 3 fraction bits: normal values (1 + f/8) 2^(e-7), subnormals
// f/8 2^-6, largest finite 448), ties to even, saturating at +-448.
inline double round_e4m3_host(double v) {
  if (v == 0.0) return v;
  const double av = std::fabs(v);
  int e;
  std::frexp(av, &e);                              // av = g 2^e, g in [0.5, 1): leading bit 2^(e-1)
  const int lead = std::max(e - 1, -6);            // below 2^-6 the spacing stays that of the subnormals
  const double q = std::ldexp(1.0, lead - 3);      // spacing of E4M3 values there
  const double r = std::min(std::nearbyint(av / q) * q, 448.0);  // default rounding: ties to even
  return std::copysign(r, v);
}

// Round the rows x cols matrix A (row-major) to E4M3 after scaling each
// column (by_row = false) or row (true) by the power of two that puts its
// largest magnitude in [224, 448), then undo the scaling.
inline void scale_round_e4m3(float* A, int rows, int cols, bool by_row) {
  const int outer = by_row ? rows : cols, inner = by_row ? cols : rows;
  for (int o = 0; o < outer; ++o) {
    auto at = [&](int i) -> float& { return by_row ? A[o * cols + i] : A[i * cols + o]; };
    double amax = 0.0;
    for (int i = 0; i < inner; ++i) amax = std::max(amax, std::fabs((double)at(i)));
    if (amax == 0.0) continue;
    int e;
    std::frexp(amax / 448.0, &e);
    for (int i = 0; i < inner; ++i)
      at(i) = (float)std::ldexp(round_e4m3_host(std::ldexp((double)at(i), -e)), e);
  }
}

template <int M>
void fill_fdm_c_args(const mg_ctx* c, int l, const float* r, FdmCArgs<M>& a) {
  constexpr int h = M / 2, ne = h + 1;
  static_assert(sizeof(FdmCArgs<M>) <= 32000, "parameter block too large");
  const LevelInfo& lv = c->lev[l];
  const float* tab = c->tab32_host.data();
  a.r = r;
  a.corr = static_cast<float*>(c->ws.corr);
  a.dinv = c->ws.tab32 + lv.dinv;
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.n = lv.n;
  a.no = lv.no[0];
  for (int d = 0; d < 3; ++d) {
    const float* S = tab + lv.t[d].S;
    const float* SW = tab + lv.t[d].SW;
    for (int t = 0; t < ne; ++t)
      for (int p = 0; p < ne; ++p) {
        a.se[d][t * ne + p] = S[t * M + p];
        a.we[d][t * ne + p] = SW[t * M + p];
      }
    for (int t = 0; t < h; ++t)
      for (int q = 0; q < h; ++q) {
        a.so[d][t * h + q] = S[t * M + ne + q];
        a.wo[d][t * h + q] = SW[t * M + ne + q];
      }
  }
  if (c->opts.fdm_operands == 1) {
    for (int d = 0; d < 3; ++d) {
      for (auto& v : a.se[d]) v = round_bf16_host(v);
      for (auto& v : a.so[d]) v = round_bf16_host(v);
      for (auto& v : a.we[d]) v = round_bf16_host(v);
      for (auto& v : a.wo[d]) v = round_bf16_host(v);
    }
  } else if (c->opts.fdm_operands == 2) {
    // FP8 with a power-of-two scale per output index: the columns p of the
    // forward halves (se[t ne + p], so[t h + q]) and the rows t of the
    // backward halves (we[t ne + p], wo[t h + q])
    for (int d = 0; d < 3; ++d) {
      scale_round_e4m3(a.se[d], ne, ne, false);
      scale_round_e4m3(a.so[d], h, h, false);
      scale_round_e4m3(a.we[d], ne, ne, true);
      scale_round_e4m3(a.wo[d], h, h, true);
    }
  }
}

template <int M>
cudaError_t launch_fdm_c_m(const mg_ctx* c, int l, const float* r) {
  using Sh = FdmCShape<M>;
  FdmCArgs<M> a;
  fill_fdm_c_args<M>(c, l, r, a);
  const int op = c->opts.fdm_operands;
  auto kern = op == 1 ? k_fdm_c<M, 1> : (op == 2 ? k_fdm_c<M, 2> : k_fdm_c<M, 0>);
  if (Sh::smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    if (e != cudaSuccess) return e;
  }
  static std::atomic<int> per_sm_cached[3] = {{0}, {0}, {0}};  // resident blocks per SM, once per variant
  int per_sm = per_sm_cached[op].load();
  if (per_sm == 0) {
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::threads, Sh::smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    per_sm_cached[op].store(per_sm);
  }
  const int64_t groups = (c->Ne + Sh::spb - 1) / Sh::spb;
  const int64_t slots = 152LL * per_sm;
  const int blocks = (int)std::min<int64_t>(groups, slots);
  launch_pdl(kern, blocks, Sh::threads, Sh::smem, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// The three kernels of the split solve, one after another on the stream.
template <int M>
cudaError_t launch_fdm_split_m(const mg_ctx* c, int l, const float* r) {
  using Sh = FdmSplitShape<M>;
  FdmCArgs<M> a;
  fill_fdm_c_args<M>(c, l, r, a);
  auto kxy = k_fdm_xy<M>;
  auto kz = k_fdm_z<M>;
  auto kyx = k_fdm_yx<M>;
  static_assert(Sh::smem <= 48 * 1024, "plane group exceeds the default shared-memory limit");
  const int64_t bp = c->Ne * Sh::groups, bz = (c->Ne * Sh::M2 + Sh::zt - 1) / Sh::zt;
  if (bp > 0x7fffffffLL || bz > 0x7fffffffLL) return cudaErrorNotSupported;
  launch_pdl(kxy, (int)bp, Sh::threads, Sh::smem, c->stream, a);
  launch_pdl(kz, (int)bz, Sh::zt, 0, c->stream, a);
  launch_pdl(kyx, (int)bp, Sh::threads, Sh::smem, c->stream, a);
  c->nlaunch += 3;
  return cudaGetLastError();
}

}  // namespace

bool fdm_c_applies(const mg_ctx* c, int l) {
  const LevelInfo& lv = c->lev[l];
  const int m = lv.m[0];
  return l >= 1 && m == lv.m[1] && m == lv.m[2] && (m & 1) && m >= 3 && m <= 35 && !c->tab32_host.empty();
}

int fdm_c_default_variant(const mg_ctx* c, int l) {
  // The split form was measured faster at every cubic width from m = 11 up,
  // also where the one-kernel form fills the SMs (16^3 mesh, m = 11: 0.55 vs
  // 0.73 ms per mixed solve; 48x8x8 mesh, m = 25: 7.1 vs 10.6 ms): its
  // kernels keep a plane or a column per thread instead of a whole tile per
  // block in shared memory.  Below m = 11 its two extra launches cost more
  // than they save.
  return fdm_c_applies(c, l) && c->lev[l].m[0] >= 11 ? 2 : 0;
}

cudaError_t launch_fdm_c(const mg_ctx* c, int l, const float* r) {
  if (!fdm_c_applies(c, l)) return cudaErrorNotSupported;
  const bool split = c->lev[l].fdm_variant == 2 && c->opts.fdm_operands == 0;
  switch (c->lev[l].m[0]) {
#define MGDG_FC(M) case M: return split ? launch_fdm_split_m<M>(c, l, r) : launch_fdm_c_m<M>(c, l, r);
    MGDG_FC(3) MGDG_FC(5) MGDG_FC(7) MGDG_FC(9) MGDG_FC(11) MGDG_FC(13) MGDG_FC(15) MGDG_FC(17) MGDG_FC(19)
    MGDG_FC(21) MGDG_FC(23) MGDG_FC(25) MGDG_FC(27) MGDG_FC(29) MGDG_FC(31) MGDG_FC(33) MGDG_FC(35)
#undef MGDG_FC
    default: return cudaErrorNotSupported;
  }
}

}  // namespace mgdg
