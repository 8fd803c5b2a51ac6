// Coarse grid solution u_0 = A_0^+ f_0 (Algorithm 1) on the P_0 = 1 level.
//
// The periodic coarse operator A_0 = Mz(x)My(x)Lx + ... is diagonalised
// exactly by the M-orthonormal eigenbases Q_d of the whole periodic 1D
// problems (L_d Q_d = M_d Q_d Lambda_d, Q_d^T M_d Q_d = I), so
//   u_0 = (Qz(x)Qy(x)Qx) (Lambda sum)^+ (Qz^T(x)Qy^T(x)Qx^T) f_0
// with the single zero eigenvalue (all three constant modes) dropped.  At
// P_0 = 1 the 1D mass matrices are (h/2) I, so every other eigenvector is
// orthogonal to the constants: dropping the constant mode is the projection
// of f_0 onto the range of A_0, and u_0 has zero Euclidean mean -- it is the
// minimum-norm solution A_0^+ f_0 without separate mean projections (they
// would change u_0 only at rounding level).  This is a direct solve: no
// iteration, no tolerance; three launches through shared memory where a
// plane and a slab of the coarse grid fit it, else six, one per axis pass.
//
// Vectors of level 0 are element-blocked with 2 nodes per direction; the
// global 1D index along x is 2 ex + i (the same for y, z).  Intermediates are
// stored in lexicographic order gx + Ngx (gy + Ngy gz).
#include <atomic>

#include "mg_internal.h"

namespace mgdg {
namespace {

struct CoarseDims {
  int Ng[3];
  int ne[3];
};

__device__ __forceinline__ int64_t eb_index(int gx, int gy, int gz, const CoarseDims& d) {
  const int ex = gx >> 1, ix = gx & 1, ey = gy >> 1, iy = gy & 1, ez = gz >> 1, iz = gz & 1;
  const int64_t e = ex + (int64_t)d.ne[0] * (ey + (int64_t)d.ne[1] * ez);
  return e * 8 + ix + 2 * (iy + 2 * iz);
}

// One-axis contraction over the lexicographic coarse grid.
//   forward: out[.. p ..] = sum_g Q[g][p] in[.. g ..]
//   backward: out[.. g ..] = sum_p Q[g][p] in[.. p ..]
// in_eb / out_eb: read / write element-blocked order instead of lexicographic.
// mean_slot >= 0: subtract scal[mean_slot] / N from every input value.
// scale: multiply each output by the pseudo-inverse of lam_x + lam_y + lam_z.
// TI / TO: type of the input / output vector (the FP32 hierarchy reads its
// right-hand side and writes its solution in FP32; intermediates are FP64).
template <typename TI, typename TO>
__device__ __forceinline__ void coarse_axis_body(BlockIdx bi_, const TI* __restrict__ in, TO* __restrict__ out,
                                                 const double* __restrict__ Q, CoarseDims d, int axis, int backward,
                                                 int in_eb, int out_eb, const double* scal, int mean_slot, int scale,
                                                 const double* lx, const double* ly, const double* lz, int nx0,
                                                 int ny0, int nz0) {
  const int Nx = d.Ng[0], Ny = d.Ng[1], Nz = d.Ng[2];
  const int64_t total = (int64_t)Nx * Ny * Nz;
  const int Na = d.Ng[axis];
  const double shift = mean_slot >= 0 ? scal[mean_slot] / (double)total : 0.0;
  // four lanes per output, each summing every fourth term, combined by
  // shuffles in a fixed order: four times the threads in flight for these
  // latency-bound passes
  const int part = threadIdx.x & 3;
  const int64_t start = (bi_.b * (int64_t)blockDim.x + threadIdx.x) >> 2;
  const int64_t stride = ((int64_t)bi_.g * blockDim.x) >> 2;
  const int64_t rounds = (total + stride - 1) / stride;  // the same for the four lanes of an output
  for (int64_t k = 0; k < rounds; ++k) {
    const int64_t idx = start + k * stride;
    const bool live = idx < total;
    int g[3] = {0, 0, 0};
    double acc = 0.0;
    if (live) {
      const int i32 = (int)idx, gyz = i32 / Nx;  // coarse sizes fit in 32 bits
      g[0] = i32 - gyz * Nx;
      g[1] = gyz % Ny;
      g[2] = gyz / Ny;
      const int o = g[axis];
      for (int t = part; t < Na; t += 4) {
        int h[3] = {g[0], g[1], g[2]};
        h[axis] = t;
        const int64_t src =
            in_eb ? eb_index(h[0], h[1], h[2], d) : h[0] + (int64_t)Nx * (h[1] + (int64_t)Ny * h[2]);
        const double q = backward ? Q[o * Na + t] : Q[t * Na + o];
        acc += q * ((double)in[src] - shift);
      }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (!live || part != 0) continue;
    if (scale) {
      if (g[0] == nx0 && g[1] == ny0 && g[2] == nz0) acc = 0.0;
      else acc /= (lx[g[0]] + ly[g[1]] + lz[g[2]]);
    }
    const int64_t dst = out_eb ? eb_index(g[0], g[1], g[2], d) : idx;
    out[dst] = (TO)acc;
  }
}

template <typename TI, typename TO>
__global__ void k_coarse_axis(const TI* __restrict__ in, TO* __restrict__ out, const double* __restrict__ Q,
                              CoarseDims d, int axis, int backward, int in_eb, int out_eb, const double* scal,
                              int mean_slot, int scale, const double* lx, const double* ly, const double* lz, int nx0,
                              int ny0, int nz0) {
  pdl_entry();
  coarse_axis_body<TI, TO>(plain_block(), in, out, Q, d, axis, backward, in_eb, out_eb, scal, mean_slot, scale, lx, ly,
                           lz, nx0, ny0, nz0);
}

// ---- the same solve in three launches, through shared memory ----
//
// The contractions along x and y couple only values of one z-plane, those
// along z only values of one y-slab, so where a plane and a slab fit shared
// memory the six passes become three kernels: x and y forward per z-plane;
// z forward, the pseudo-inverse of the eigenvalue sums and z backward per
// y-slab; y and x backward per z-plane.  Each plane or slab is split into
// `chunks` pieces over as many blocks (x-columns for the first two kernels,
// y-rows for the last), so that the FP64 work spreads over the SMs; no
// product is computed twice.  Each output is one sequential sum over the
// contracted index.
struct CoarseFused {
  const double* Q[3];
  const double* lam[3];
  CoarseDims d;
  int null_mode[3];
  const double* scal;
  int mean_slot;
  int chunks[3];  // pieces per plane (x then y forward), slab (z), plane (y then x backward)
};

__device__ __forceinline__ void chunk_range(int n, int chunks, int ch, int* lo, int* hi) {
  const int w = (n + chunks - 1) / chunks;
  *lo = ch * w;
  *hi = *lo + w < n ? *lo + w : n;
}

template <typename TI>
__device__ __forceinline__ void coarse_xy_body(BlockIdx bi_, const TI* __restrict__ in, double* __restrict__ out,
                                               CoarseFused a) {
  extern __shared__ __align__(16) double cf_sm[];
  const int Nx = a.d.Ng[0], Ny = a.d.Ng[1], Nz = a.d.Ng[2], plane = Nx * Ny, C = a.chunks[0];
  double* P = cf_sm;
  double* T = cf_sm + plane;
  const double shift = a.mean_slot >= 0 ? a.scal[a.mean_slot] / ((double)plane * Nz) : 0.0;
  const double* __restrict__ Qx = a.Q[0];
  const double* __restrict__ Qy = a.Q[1];
  for (int vb = bi_.b; vb < Nz * C; vb += bi_.g) {
    const int gz = vb / C;
    int p0, p1;
    chunk_range(Nx, C, vb - gz * C, &p0, &p1);
    const int w = p1 - p0;
    for (int i = threadIdx.x; i < plane; i += blockDim.x) {
      const int gx = i % Nx, gy = i / Nx;
      P[i] = (double)in[eb_index(gx, gy, gz, a.d)] - shift;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < w * Ny; i += blockDim.x) {  // x forward, columns p0 .. p1 - 1
      const int p = p0 + i % w, gy = i / w;
      double acc = 0.0;
      for (int t = 0; t < Nx; ++t) acc += Qx[t * Nx + p] * P[t + Nx * gy];
      T[p + Nx * gy] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < w * Ny; i += blockDim.x) {  // y forward, the same columns
      const int p = p0 + i % w, q = i / w;
      double acc = 0.0;
      for (int t = 0; t < Ny; ++t) acc += Qy[t * Ny + q] * T[p + Nx * t];
      out[p + Nx * q + (int64_t)plane * gz] = acc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void coarse_z_body(BlockIdx bi_, double* __restrict__ A, CoarseFused a) {
  extern __shared__ __align__(16) double cf_sm[];
  const int Nx = a.d.Ng[0], Ny = a.d.Ng[1], Nz = a.d.Ng[2], slab = Nx * Nz, C = a.chunks[1];
  double* S = cf_sm;
  double* V = cf_sm + slab;
  const double* __restrict__ Qz = a.Q[2];
  for (int vb = bi_.b; vb < Ny * C; vb += bi_.g) {
    const int gy = vb / C;
    int x0, x1;
    chunk_range(Nx, C, vb - gy * C, &x0, &x1);
    const int w = x1 - x0;
    for (int i = threadIdx.x; i < w * Nz; i += blockDim.x) {  // the chunk's columns of the slab
      const int gx = x0 + i % w, gz = i / w;
      S[gx + Nx * gz] = A[gx + (int64_t)Nx * (gy + (int64_t)Ny * gz)];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < w * Nz; i += blockDim.x) {  // z forward, pseudo-inverse
      const int gx = x0 + i % w, r = i / w;
      double acc = 0.0;
      for (int t = 0; t < Nz; ++t) acc += Qz[t * Nz + r] * S[gx + Nx * t];
      if (gx == a.null_mode[0] && gy == a.null_mode[1] && r == a.null_mode[2]) acc = 0.0;
      else acc /= (a.lam[0][gx] + a.lam[1][gy] + a.lam[2][r]);
      V[gx + Nx * r] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < w * Nz; i += blockDim.x) {  // z backward
      const int gx = x0 + i % w, gz = i / w;
      double acc = 0.0;
      for (int t = 0; t < Nz; ++t) acc += Qz[gz * Nz + t] * V[gx + Nx * t];
      A[gx + (int64_t)Nx * (gy + (int64_t)Ny * gz)] = acc;
    }
    __syncthreads();
  }
}

template <typename TO>
__device__ __forceinline__ void coarse_yx_body(BlockIdx bi_, const double* __restrict__ A, TO* __restrict__ out,
                                               CoarseFused a) {
  extern __shared__ __align__(16) double cf_sm[];
  const int Nx = a.d.Ng[0], Ny = a.d.Ng[1], Nz = a.d.Ng[2], plane = Nx * Ny, C = a.chunks[2];
  double* P = cf_sm;
  double* T = cf_sm + plane;
  const double* __restrict__ Qx = a.Q[0];
  const double* __restrict__ Qy = a.Q[1];
  for (int vb = bi_.b; vb < Nz * C; vb += bi_.g) {
    const int gz = vb / C;
    int y0, y1;
    chunk_range(Ny, C, vb - gz * C, &y0, &y1);
    const int h = y1 - y0;
    for (int i = threadIdx.x; i < plane; i += blockDim.x) P[i] = A[i + (int64_t)plane * gz];
    __syncthreads();
    for (int i = threadIdx.x; i < Nx * h; i += blockDim.x) {  // y backward, rows y0 .. y1 - 1
      const int gx = i % Nx, gy = y0 + i / Nx;
      double acc = 0.0;
      for (int t = 0; t < Ny; ++t) acc += Qy[gy * Ny + t] * P[gx + Nx * t];
      T[gx + Nx * gy] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Nx * h; i += blockDim.x) {  // x backward, element-blocked result
      const int gx = i % Nx, gy = y0 + i / Nx;
      double acc = 0.0;
      for (int t = 0; t < Nx; ++t) acc += Qx[gx * Nx + t] * T[t + Nx * gy];
      out[eb_index(gx, gy, gz, a.d)] = (TO)acc;
    }
    __syncthreads();
  }
}

template <typename TI>
__global__ void __launch_bounds__(256) k_coarse_xy(const TI* __restrict__ in, double* __restrict__ out,
                                                   const __grid_constant__ CoarseFused a) {
  pdl_entry();
  coarse_xy_body<TI>(plain_block(), in, out, a);
}

__global__ void __launch_bounds__(256) k_coarse_z(double* __restrict__ A, const __grid_constant__ CoarseFused a) {
  pdl_entry();
  coarse_z_body(plain_block(), A, a);
}

template <typename TO>
__global__ void __launch_bounds__(256) k_coarse_yx(const double* __restrict__ A, TO* __restrict__ out,
                                                   const __grid_constant__ CoarseFused a) {
  pdl_entry();
  coarse_yx_body<TO>(plain_block(), A, out, a);
}

// Shared memory of the three kernels (two planes or two slabs of FP64),
// rounded up to 16 KB so that batched problems of similar coarse grids merge
// their launches (records merge only at equal shared memory), or 0 if a
// plane or slab does not fit (then the six passes).  Measured against the six
// passes: 16^3 mesh 0.42 vs 0.63 ms per FP64 solve (12 coarse solves), 16
// small problems batched 22.6 vs 23.9 ms.
inline size_t coarse_fused_smem(const CoarseDims& d) {
  const size_t plane = (size_t)d.Ng[0] * d.Ng[1], slab = (size_t)d.Ng[0] * d.Ng[2];
  const size_t bytes = 2 * sizeof(double) * (plane > slab ? plane : slab);
  const size_t step = 16 * 1024, rounded = (bytes + step - 1) / step * step;
  return rounded <= 96 * 1024 ? rounded : 0;
}

template <typename TI, typename TO>
cudaError_t coarse_fused(const CoarseFused& a, const TI* f0, double* A, TO* u0, size_t smem, cudaStream_t s) {
  static std::atomic<size_t> set_xy{48 * 1024}, set_z{48 * 1024}, set_yx{48 * 1024};
  cudaError_t e;
  if ((e = allow_smem((const void*)k_coarse_xy<TI>, smem, set_xy)) != cudaSuccess) return e;
  if ((e = allow_smem((const void*)k_coarse_z, smem, set_z)) != cudaSuccess) return e;
  if ((e = allow_smem((const void*)k_coarse_yx<TO>, smem, set_yx)) != cudaSuccess) return e;
  const int vb[3] = {a.d.Ng[2] * a.chunks[0], a.d.Ng[1] * a.chunks[1], a.d.Ng[2] * a.chunks[2]};
  int nb[3];
  for (int k = 0; k < 3; ++k) nb[k] = vb[k] < 152 * 8 ? vb[k] : 152 * 8;
  launch_pdl<&coarse_xy_body<TI>>(k_coarse_xy<TI>, nb[0], 256, smem, s, f0, A, a);
  launch_pdl<&coarse_z_body>(k_coarse_z, nb[1], 256, smem, s, A, a);
  launch_pdl<&coarse_yx_body<TO>>(k_coarse_yx<TO>, nb[2], 256, smem, s, A, u0, a);
  return cudaGetLastError();
}

// One axis pass (k_coarse_axis, or its grouped twin's body when Twin).
template <bool Twin, typename TI, typename TO>
void axis_pass(int blocks, cudaStream_t s, const TI* in, TO* out, const double* Q, const CoarseDims& d, int axis,
               int backward, int in_eb, int out_eb, const double* scal, int mean_slot, int scale,
               const double* lx = nullptr, const double* ly = nullptr, const double* lz = nullptr, int nx0 = 0,
               int ny0 = 0, int nz0 = 0) {
  launch_pdl<Twin ? &coarse_axis_body<TI, TO> : nullptr>(k_coarse_axis<TI, TO>, blocks, 256, 0, s, in, out, Q, d,
                                                         axis, backward, in_eb, out_eb, scal, mean_slot, scale, lx,
                                                         ly, lz, nx0, ny0, nz0);
}

// The six axis passes: f0 (element-blocked) -> x, y, z forward, scale, z, y, x
// backward -> u0 (element-blocked); A, B lexicographic FP64 scratch.
template <typename TI, typename TO>
cudaError_t coarse_passes(const double* const Q[3], const double* const lam[3], const CoarseDims& d,
                          const int null_mode[3], const TI* f0, double* A, double* B, TO* u0, const double* scal,
                          int mean_slot, cudaStream_t s) {
  const int64_t N0 = (int64_t)d.Ng[0] * d.Ng[1] * d.Ng[2];
  int64_t blocks = (4 * N0 + 255) / 256;  // four lanes per output
  if (blocks > 152 * 8) blocks = 152 * 8;
  const int* nz = null_mode;
  const int b = (int)blocks;
  // the FP32 / double-float hierarchies' coarse solves run through the grouped
  // twins (batched solves), the FP64 hierarchy's through the plain kernels
  constexpr bool kTwin = kTwinType<TI> || kTwinType<TO>;
  axis_pass<kTwin>(b, s, f0, A, Q[0], d, 0, 0, 1, 0, scal, mean_slot, 0);
  axis_pass<kTwin>(b, s, A, B, Q[1], d, 1, 0, 0, 0, scal, -1, 0);
  axis_pass<kTwin>(b, s, B, A, Q[2], d, 2, 0, 0, 0, scal, -1, 1, lam[0], lam[1], lam[2], nz[0], nz[1], nz[2]);
  axis_pass<kTwin>(b, s, A, B, Q[2], d, 2, 1, 0, 0, scal, -1, 0);
  axis_pass<kTwin>(b, s, B, A, Q[1], d, 1, 1, 0, 0, scal, -1, 0);
  axis_pass<kTwin>(b, s, A, u0, Q[0], d, 0, 1, 0, 1, scal, -1, 0);
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t coarse_solve_t(const mg_ctx* c, const TI* f0, TO* u0) {
  const LevelInfo& lv = c->lev[0];
  CoarseDims d;
  for (int k = 0; k < 3; ++k) {
    d.Ng[k] = c->Ng[k];
    d.ne[k] = c->ne[k];
  }
  const double* tab = c->ws.tab64;
  const double* Q[3] = {tab + lv.t[0].Q, tab + lv.t[1].Q, tab + lv.t[2].Q};
  const double* lam[3] = {tab + lv.t[0].qlam, tab + lv.t[1].qlam, tab + lv.t[2].qlam};
  const size_t smem = coarse_fused_smem(d);
  if (smem > 0) {
    CoarseFused a;
    for (int k = 0; k < 3; ++k) {
      a.Q[k] = Q[k];
      a.lam[k] = lam[k];
      a.null_mode[k] = c->coarse_null[k];
    }
    a.d = d;
    a.scal = c->ws.scal;
    a.mean_slot = -1;
    // pieces per plane / slab: about two blocks per SM in all, each piece at
    // least 4 columns or rows wide
    const int outer[3] = {d.Ng[2], d.Ng[1], d.Ng[2]}, width[3] = {d.Ng[0], d.Ng[0], d.Ng[1]};
    for (int k = 0; k < 3; ++k) {
      const int want = (2 * 152 + outer[k] - 1) / outer[k], most = (width[k] + 3) / 4;
      a.chunks[k] = want < most ? want : most;
      if (a.chunks[k] < 1) a.chunks[k] = 1;
    }
    c->nlaunch += 3;
    return coarse_fused<TI, TO>(a, f0, c->ws.coarse_a, u0, smem, c->stream);
  }
  c->nlaunch += 6;
  return coarse_passes<TI, TO>(Q, lam, d, c->coarse_null, f0, c->ws.coarse_a, c->ws.coarse_b, u0, c->ws.scal, -1,
                               c->stream);
}

}  // namespace

// Graded mesh: the level-0 mass is not a multiple of I, so the eigenbases are
// not orthogonal to the constants in the Euclidean sense.  Dropping the
// constant mode then neither projects f0 onto the range of A_0 nor gives the
// zero-mean solution: both become explicit passes (f0 - mean(f0) into the
// FP64 scratch coarse_f, and u0 - mean(u0) at the end).
template <typename T>
cudaError_t graded_coarse_solve(const mg_ctx* c, const T* f0, T* u0) {
  cudaError_t e = launch_gcenter<T>(c, f0, c->ws.coarse_f);
  if (e == cudaSuccess) e = coarse_solve_t<double, T>(c, c->ws.coarse_f, u0);
  if (e == cudaSuccess) e = launch_gmean_zero<T>(c, u0);
  return e;
}

cudaError_t launch_coarse_solve(const mg_ctx* c, const double* f0, double* u0) {
  if (c->graded) return graded_coarse_solve<double>(c, f0, u0);
  return coarse_solve_t<double, double>(c, f0, u0);
}

cudaError_t launch_coarse_fdm_raw(const double* const Q[3], const double* const lam[3], const int Ng[3],
                                  const int ne[3], const int null_mode[3], const double* f0, double* A, double* B,
                                  double* u0, const double* scal, int mean_slot, cudaStream_t s) {
  CoarseDims d;
  for (int k = 0; k < 3; ++k) {
    d.Ng[k] = Ng[k];
    d.ne[k] = ne[k];
  }
  return coarse_passes<double, double>(Q, lam, d, null_mode, f0, A, B, u0, scal, mean_slot, s);
}

cudaError_t launch_coarse_solve_df64(const mg_ctx* c, const df64* f0, df64* u0) {
  return coarse_solve_t<df64, df64>(c, f0, u0);
}

cudaError_t launch_coarse_solve_f32(const mg_ctx* c, const float* f0, float* u0) {
  // The coarsest solve of the FP32 hierarchy runs in FP64: the first pass
  // reads the FP32 right-hand side, the last writes the FP32 solution.
  if (c->graded) return graded_coarse_solve<float>(c, f0, u0);
  return coarse_solve_t<float, float>(c, f0, u0);
}

}  // namespace mgdg
