// Fast-diagonalisation smoother kernel with the subdomain width m as a
// compile-time constant (Section 3.1): the 1D lines live in registers and the
// even/odd products are fully unrolled.  Same algorithm, same memory layout
// and same results as the run-time-size kernel in schwarz.cu; included only by
// the instantiation units fdm_m_*.cu.
#pragma once

#include "mg_internal.h"

namespace mgdg {

template <typename T>
struct FdmArgs {
  const T* tab;
  const T* r;
  T* corr;
  int64_t Ne;
  int nx, ny, nz, n, m, no, spb;  // m, no: cubic subdomains (compile-time kernel)
  int md[3], nod[3];              // per-direction width and layers (run-time kernel)
  int s_in_smem;                  // run-time kernel: 1D factors staged in shared memory
  int64_t S[3], SW[3], dinv;
};

__device__ __forceinline__ void fdm_sub_node(int a, int n, int no, int* de, int* ii) {
  if (a < no) { *de = -1; *ii = n - no + a; }
  else if (a < no + n) { *de = 0; *ii = a - no; }
  else { *de = 1; *ii = a - no - n; }
}

__device__ __forceinline__ int fdm_wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// y = S^T x for a reflection-symmetric line (even modes first); x is overwritten.
template <typename T, int M>
__device__ __forceinline__ void fdm_fwd(T (&x)[M], const T* __restrict__ S, T (&y)[M]) {
  constexpr int h = M / 2, ne = h + 1;
#pragma unroll
  for (int a = 0; a < h; ++a) {
    const T xa = x[a], xb = x[M - 1 - a];
    x[a] = xa + xb;
    x[M - 1 - a] = xa - xb;
  }
#pragma unroll
  for (int p = 0; p < ne; ++p) {
    Acc<T> acc;
    acc.init(S[p], x[0]);
#pragma unroll
    for (int a = 1; a <= h; ++a) acc.add(S[a * M + p], x[a]);
    y[p] = acc.get();
  }
#pragma unroll
  for (int q = 0; q < h; ++q) {
    Acc<T> acc;
    acc.init(S[ne + q], x[M - 1]);
#pragma unroll
    for (int a = 1; a < h; ++a) acc.add(S[a * M + ne + q], x[M - 1 - a]);
    y[ne + q] = acc.get();
  }
}

// x = SW v (weights folded into SW).
template <typename T, int M>
__device__ __forceinline__ void fdm_bwd(const T (&v)[M], const T* __restrict__ SW, T (&x)[M]) {
  constexpr int h = M / 2, ne = h + 1;
#pragma unroll
  for (int a = 0; a <= h; ++a) {
    Acc<T> ea;
    ea.init(SW[a * M], v[0]);
#pragma unroll
    for (int p = 1; p < ne; ++p) ea.add(SW[a * M + p], v[p]);
    const T E = ea.get();
    if (a < h) {
      Acc<T> oa;
      oa.init(SW[a * M + ne], v[ne]);
#pragma unroll
      for (int q = 1; q < h; ++q) oa.add(SW[a * M + ne + q], v[ne + q]);
      const T O = oa.get();
      x[a] = E + O;
      x[M - 1 - a] = E - O;
    } else {
      x[a] = E;
    }
  }
}

// The same two products with the output loop rolled, each output written to
// out[i * os] as soon as it is formed: the double-float pair arithmetic makes
// the fully unrolled form too large for the instruction cache (the same
// operations in the same order, so the same results).
template <typename T, int M>
__device__ __forceinline__ void fdm_fwd_rolled(T (&x)[M], const T* __restrict__ S, T* out, int os) {
  constexpr int h = M / 2, ne = h + 1;
#pragma unroll
  for (int a = 0; a < h; ++a) {
    const T xa = x[a], xb = x[M - 1 - a];
    x[a] = xa + xb;
    x[M - 1 - a] = xa - xb;
  }
#pragma unroll 1
  for (int p = 0; p < ne; ++p) {
    Acc<T> acc;
    acc.init(S[p], x[0]);
#pragma unroll
    for (int a = 1; a <= h; ++a) acc.add(S[a * M + p], x[a]);
    out[p * os] = acc.get();
  }
#pragma unroll 1
  for (int q = 0; q < h; ++q) {
    Acc<T> acc;
    acc.init(S[ne + q], x[M - 1]);
#pragma unroll
    for (int a = 1; a < h; ++a) acc.add(S[a * M + ne + q], x[M - 1 - a]);
    out[(ne + q) * os] = acc.get();
  }
}

template <typename T, int M>
__device__ __forceinline__ void fdm_bwd_rolled(const T (&v)[M], const T* __restrict__ SW, T* out, int os) {
  constexpr int h = M / 2, ne = h + 1;
#pragma unroll 1
  for (int a = 0; a <= h; ++a) {
    Acc<T> ea;
    ea.init(SW[a * M], v[0]);
#pragma unroll
    for (int p = 1; p < ne; ++p) ea.add(SW[a * M + p], v[p]);
    const T E = ea.get();
    if (a < h) {
      Acc<T> oa;
      oa.init(SW[a * M + ne], v[ne]);
#pragma unroll
      for (int q = 1; q < h; ++q) oa.add(SW[a * M + ne + q], v[ne + q]);
      const T O = oa.get();
      out[a * os] = E + O;
      out[(M - 1 - a) * os] = E - O;
    } else {
      out[a * os] = E;
    }
  }
}

// Line transforms of the smoother passes: out[i * os] = (S^T x)_i, resp. (SW v)_i.
template <typename T, int M>
__device__ __forceinline__ void line_fwd(T (&x)[M], const T* __restrict__ S, T* out, int os) {
  if constexpr (std::is_same<T, df64>::value) {
    fdm_fwd_rolled<T, M>(x, S, out, os);
  } else {
    T y[M];
    fdm_fwd<T, M>(x, S, y);
#pragma unroll
    for (int p = 0; p < M; ++p) out[p * os] = y[p];
  }
}

template <typename T, int M>
__device__ __forceinline__ void line_bwd(const T (&v)[M], const T* __restrict__ SW, T* out, int os) {
  if constexpr (std::is_same<T, df64>::value) {
    fdm_bwd_rolled<T, M>(v, SW, out, os);
  } else {
    T x[M];
    fdm_bwd<T, M>(v, SW, x);
#pragma unroll
    for (int p = 0; p < M; ++p) out[p * os] = x[p];
  }
}

// Subdomains per block and whether their tiles fit in shared memory (the
// last pass always writes the corrections to the global buffer).
template <typename T, int M>
struct FdmShape {
  // subdomains per block: one from m = 11 up; about 256 lines a pass below
  static constexpr int spb = M * M >= 100 ? 1 : 256 / (M * M);
  static constexpr size_t table_bytes = sizeof(T) * 6 * M * M;
  static constexpr size_t tile_bytes = sizeof(T) * spb * M * M * M;
  static constexpr bool smem_tile = table_bytes + tile_bytes <= 210 * 1024;
  static constexpr size_t smem = table_bytes + (smem_tile ? tile_bytes : 0);
};

template <typename T, int M>
__device__ __forceinline__ void fdm_m_body(BlockIdx bi_, FdmArgs<T> a) {
  constexpr int M2 = M * M, M3 = M2 * M;
  constexpr bool kSmemTile = FdmShape<T, M>::smem_tile;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sS = reinterpret_cast<T*>(smraw);  // 3 M^2
  T* sSW = sS + 3 * M2;                 // 3 M^2
  T* sTile = sSW + 3 * M2;              // spb M^3 (if kSmemTile)
  for (int i = threadIdx.x; i < M2; i += blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      sS[d * M2 + i] = a.tab[a.S[d] + i];
      sSW[d * M2 + i] = a.tab[a.SW[d] + i];
    }
  }
  __syncthreads();
  const T* __restrict__ dinv = a.tab + a.dinv;
  const int n = a.n, no = a.no, n3 = n * n * n, spb = a.spb;
  const int lines = spb * M2;
  for (int64_t s0 = (int64_t)bi_.b * spb; s0 < a.Ne; s0 += (int64_t)bi_.g * spb) {
    // pass 1: gather x-lines of r_s and transform (forward, x)
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int64_t s = s0 + ln / M2;
      if (s >= a.Ne) continue;
      const int l2 = ln % M2, b = l2 % M, c = l2 / M;
      const int s32 = (int)s, sxy = s32 / a.nx;  // element indices fit in 32 bits
      const int sx = s32 - sxy * a.nx, sy = sxy % a.ny, sz = sxy / a.ny;
      int dy, iy, dz, iz;
      fdm_sub_node(b, n, no, &dy, &iy);
      fdm_sub_node(c, n, no, &dz, &iz);
      const int64_t row = a.nx * (fdm_wrap(sy + dy, a.ny) + (int64_t)a.ny * fdm_wrap(sz + dz, a.nz));
      const int loc = n * (iy + n * iz);
      // offsets of position t of the line in the left / centre / right element
      const int64_t ol = (fdm_wrap(sx - 1, a.nx) + row) * n3 + loc + (n - no);
      const int64_t oc = (sx + row) * n3 + loc - no;
      const int64_t orr = (fdm_wrap(sx + 1, a.nx) + row) * n3 + loc - (no + n);
      T x[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = a.r[(t < no ? ol : (t < no + n ? oc : orr)) + t];
      T* tile = (kSmemTile ? sTile + (ln / M2) * M3 : a.corr + s * (int64_t)M3) + M * l2;
      line_fwd<T, M>(x, sS, tile, 1);
    }
    __syncthreads();
    // pass 2: forward, y
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int64_t s = s0 + ln / M2;
      if (s >= a.Ne) continue;
      const int l2 = ln % M2;
      T* line = (kSmemTile ? sTile + (ln / M2) * M3 : a.corr + s * (int64_t)M3) + (l2 % M) + M2 * (l2 / M);
      T x[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = line[t * M];
      line_fwd<T, M>(x, sS + M2, line, M);
    }
    __syncthreads();
    // pass 3: forward z, scale by 1 / (lam_x + lam_y + lam_z), backward z
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int64_t s = s0 + ln / M2;
      if (s >= a.Ne) continue;
      const int l2 = ln % M2;
      T* line = (kSmemTile ? sTile + (ln / M2) * M3 : a.corr + s * (int64_t)M3) + l2;
      T x[M], y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = line[t * M2];
      if constexpr (std::is_same<T, df64>::value) {  // through the tile (rolled products)
        fdm_fwd_rolled<T, M>(x, sS + 2 * M2, line, M2);
#pragma unroll
        for (int t = 0; t < M; ++t) y[t] = line[t * M2] * dinv[l2 + t * M2];
      } else {
        fdm_fwd<T, M>(x, sS + 2 * M2, y);
#pragma unroll
        for (int t = 0; t < M; ++t) y[t] *= dinv[l2 + t * M2];
      }
      line_bwd<T, M>(y, sSW + 2 * M2, line, M2);
    }
    __syncthreads();
    // pass 4: backward, y
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int64_t s = s0 + ln / M2;
      if (s >= a.Ne) continue;
      const int l2 = ln % M2;
      T* line = (kSmemTile ? sTile + (ln / M2) * M3 : a.corr + s * (int64_t)M3) + (l2 % M) + M2 * (l2 / M);
      T y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) y[t] = line[t * M];
      line_bwd<T, M>(y, sSW + M2, line, M);
    }
    __syncthreads();
    // pass 5: backward, x (weights folded into SW)
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int64_t s = s0 + ln / M2;
      if (s >= a.Ne) continue;
      const int l2 = ln % M2;
      const T* line = (kSmemTile ? sTile + (ln / M2) * M3 : a.corr + s * (int64_t)M3) + M * l2;
      T* outl = a.corr + s * (int64_t)M3 + M * l2;
      T y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) y[t] = line[t];
      line_bwd<T, M>(y, sSW, outl, 1);
    }
    __syncthreads();
  }
}

template <typename T, int M>
__global__ void __launch_bounds__(256) k_fdm_m(FdmArgs<T> a) {
  pdl_entry();
  fdm_m_body<T, M>(plain_block(), a);
}

template <typename T, int M>
cudaError_t launch_fdm_m(const FdmArgs<T>& a, int blocks, int threads, size_t /*smem*/, cudaStream_t s) {
  const size_t smem = FdmShape<T, M>::smem;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fdm_m<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  launch_pdl<fdm_m_body<T, M>>(k_fdm_m<T, M>, blocks, threads, smem, s, a);  // with its grouped twin
  return cudaGetLastError();
}

#define MGDG_FDM_EXTERN(M)                                                                                   \
  extern template cudaError_t launch_fdm_m<double, M>(const FdmArgs<double>&, int, int, size_t, cudaStream_t); \
  extern template cudaError_t launch_fdm_m<float, M>(const FdmArgs<float>&, int, int, size_t, cudaStream_t);

#define MGDG_FDM_INSTANTIATE(M)                                                                              \
  template cudaError_t launch_fdm_m<double, M>(const FdmArgs<double>&, int, int, size_t, cudaStream_t);     \
  template cudaError_t launch_fdm_m<float, M>(const FdmArgs<float>&, int, int, size_t, cudaStream_t);

// Double-float instantiations exist for the widths of N_O = 1, 2 up to P = 16
// (other widths use the run-time-size kernel).
#define MGDG_FDM_DF_WIDTHS(X) X(3) X(5) X(7) X(9) X(11) X(13) X(17) X(19) X(21)
#define MGDG_FDM_EXTERN_DF(M) \
  extern template cudaError_t launch_fdm_m<df64, M>(const FdmArgs<df64>&, int, int, size_t, cudaStream_t);
#define MGDG_FDM_INSTANTIATE_DF(M) \
  template cudaError_t launch_fdm_m<df64, M>(const FdmArgs<df64>&, int, int, size_t, cudaStream_t);

}  // namespace mgdg
