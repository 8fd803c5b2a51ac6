// Graded-mesh smoother with compile-time subdomain widths (odd m = 3 .. 25).
//
// The same gather and fast diagonalisation as the run-time-width kernel of
// graded.cu (Section 3.1: du_s = (Sz (x) Sy (x) Sx) D^-1 (Sz^T (x) Sy^T (x)
// Sx^T) R_s r with the eigenbases of the three lines through the subdomain's
// element), arranged like the uniform compile-time smoother: a thread keeps
// one subdomain line in registers, the tile stays in shared memory between
// the passes (only the last pass writes the correction buffer), and small
// widths put several subdomains in one block.  A graded subdomain line has no
// reflection symmetry, so each 1D product is the whole m x m product; each
// subdomain stages its own factors (S, SW and lam of its three lines) in
// shared memory.
#include <algorithm>
#include <type_traits>

#include "mg_internal.h"

namespace mgdg {
namespace {

template <typename T>
const T* gtab(const mg_ctx* c);
template <>
const double* gtab<double>(const mg_ctx* c) { return c->ws.tab64; }
template <>
const float* gtab<float>(const mg_ctx* c) { return c->ws.tab32; }

__device__ __forceinline__ int gw(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// Subdomain position a -> (element offset -1 / 0 / +1, node index in that element).
__device__ __forceinline__ void fdm_sub_node_g(int a, int n, int no, int* de, int* ii) {
  if (a < no) { *de = -1; *ii = n - no + a; }
  else if (a < no + n) { *de = 0; *ii = a - no; }
  else { *de = 1; *ii = a - no - n; }
}

template <typename T>
struct GFdmMArgs {
  const T* tab;
  const T* r;
  T* corr;
  int64_t Ne;
  int nx, ny, nz, n, no, spb;
  int64_t S[3], SW[3], lam[3];
};

template <typename T, int M>
struct GShape {
  static constexpr int spb = M * M >= 100 ? 1 : 256 / (M * M);
  // row stride of the staged factors: FP32 rows padded to a multiple of four
  // (zeros) for 16-byte shared-memory loads, FP64 rows unpadded
  static constexpr int RS = std::is_same<T, float>::value ? (M + 3) / 4 * 4 : M;
  static constexpr int MR = M * RS;                                  // one staged factor
  static constexpr size_t table_vals = 6 * MR + (3 * M + 3) / 4 * 4;  // per subdomain: S, SW, lam of three lines
  static constexpr size_t table_bytes = sizeof(T) * spb * table_vals;
  static constexpr size_t tile_bytes = sizeof(T) * spb * M * M * M;
  static constexpr bool smem_tile = table_bytes + tile_bytes <= 200 * 1024;
  static constexpr size_t smem = table_bytes + (smem_tile ? tile_bytes : 0);
};

// y_p = sum_a S[a][p] x_a (S staged with row stride RS)
template <typename T, int M>
__device__ __forceinline__ void gfwd_reg(const T (&x)[M], const T* __restrict__ S, T (&y)[M]) {
  constexpr int RS = GShape<T, M>::RS;
  if constexpr (std::is_same<T, float>::value) {
    // four outputs per 16-byte load of a factor row
#pragma unroll
    for (int g = 0; g < RS / 4; ++g) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int a = 0; a < M; ++a) {
        const float4 s4 = *reinterpret_cast<const float4*>(S + a * RS + 4 * g);
        acc.x += s4.x * x[a];
        acc.y += s4.y * x[a];
        acc.z += s4.z * x[a];
        acc.w += s4.w * x[a];
      }
      y[4 * g] = acc.x;
      if (4 * g + 1 < M) y[4 * g + 1 < M ? 4 * g + 1 : 0] = acc.y;
      if (4 * g + 2 < M) y[4 * g + 2 < M ? 4 * g + 2 : 0] = acc.z;
      if (4 * g + 3 < M) y[4 * g + 3 < M ? 4 * g + 3 : 0] = acc.w;
    }
  } else {
#pragma unroll
    for (int p = 0; p < M; ++p) {
      T acc = S[p] * x[0];
#pragma unroll
      for (int a = 1; a < M; ++a) acc += S[a * RS + p] * x[a];
      y[p] = acc;
    }
  }
}

// y_p = sum_a S[a][p] x_a, written to out[p * os]
template <typename T, int M>
__device__ __forceinline__ void gfwd(const T (&x)[M], const T* __restrict__ S, T* out, int os) {
  if constexpr (std::is_same<T, float>::value) {
    T y[M];
    gfwd_reg<T, M>(x, S, y);
#pragma unroll
    for (int p = 0; p < M; ++p) out[p * os] = y[p];
  } else {
    // each output stored as soon as it is formed (fewer live registers)
#pragma unroll
    for (int p = 0; p < M; ++p) {
      T acc = S[p] * x[0];
#pragma unroll
      for (int a = 1; a < M; ++a) acc += S[a * M + p] * x[a];
      out[p * os] = acc;
    }
  }
}

// x_a = sum_p SW[a][p] v_p, written to out[a * os]
template <typename T, int M>
__device__ __forceinline__ void gbwd(const T (&v)[M], const T* __restrict__ SW, T* out, int os) {
  constexpr int RS = GShape<T, M>::RS;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    T acc = 0;
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
      for (int g = 0; g < RS / 4; ++g) {
        const float4 s4 = *reinterpret_cast<const float4*>(SW + a * RS + 4 * g);
        acc += s4.x * v[4 * g];
        if (4 * g + 1 < M) acc += s4.y * v[4 * g + 1 < M ? 4 * g + 1 : 0];
        if (4 * g + 2 < M) acc += s4.z * v[4 * g + 2 < M ? 4 * g + 2 : 0];
        if (4 * g + 3 < M) acc += s4.w * v[4 * g + 3 < M ? 4 * g + 3 : 0];
      }
    } else {
      acc = SW[a * RS] * v[0];
#pragma unroll
      for (int p = 1; p < M; ++p) acc += SW[a * RS + p] * v[p];
    }
    out[a * os] = acc;
  }
}

template <typename T, int M>
__global__ void __launch_bounds__(256) k_gfdm_m(GFdmMArgs<T> a) {
  pdl_entry();
  constexpr int M2 = M * M, M3 = M2 * M;
  constexpr int RS = GShape<T, M>::RS, MR = GShape<T, M>::MR;
  constexpr int TV = (int)GShape<T, M>::table_vals;
  constexpr bool kSmemTile = GShape<T, M>::smem_tile;
  extern __shared__ __align__(16) unsigned char gm_raw[];
  T* sTab = reinterpret_cast<T*>(gm_raw);  // spb x (S[3], SW[3] with row stride RS, lam[3])
  T* sTile = sTab + a.spb * TV;            // spb M^3 (if kSmemTile)
  const int n = a.n, no = a.no, n3 = n * n * n, spb = a.spb;
  const int lines = spb * M2;
  for (int64_t s0 = (int64_t)blockIdx.x * spb; s0 < a.Ne; s0 += (int64_t)gridDim.x * spb) {
    // factors of the group's subdomains
    for (int i = threadIdx.x; i < spb * TV; i += blockDim.x) {
      const int k = i / TV, q = i - k * TV;
      const int64_t s = s0 + k;
      if (s >= a.Ne) continue;
      const int s32 = (int)s, sxy = s32 / a.nx;
      const int lx = s32 - sxy * a.nx, ly = sxy % a.ny, lz = sxy / a.ny;
      T v = 0;
      if (q < 6 * MR) {
        const int d = q / (2 * MR), r = q - d * 2 * MR;
        const int wsw = r >= MR, rr = r - wsw * MR, row = rr / RS, col = rr - row * RS;
        const int64_t ld = d == 0 ? lx : (d == 1 ? ly : lz);
        if (col < M) {
          const int64_t base = wsw ? (d == 0 ? a.SW[0] : (d == 1 ? a.SW[1] : a.SW[2]))
                                   : (d == 0 ? a.S[0] : (d == 1 ? a.S[1] : a.S[2]));
          v = a.tab[base + ld * M2 + row * M + col];
        }
      } else if (q < 6 * MR + 3 * M) {
        const int d = (q - 6 * MR) / M, r = (q - 6 * MR) - d * M;
        const int64_t ld = d == 0 ? lx : (d == 1 ? ly : lz);
        v = a.tab[(d == 0 ? a.lam[0] : (d == 1 ? a.lam[1] : a.lam[2])) + ld * M + r];
      }
      sTab[i] = v;
    }
    __syncthreads();
    // pass 1: gather the x-lines of r_s = R_s r, forward along x
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int k = ln / M2;
      const int64_t s = s0 + k;
      if (s >= a.Ne) continue;
      const int l2 = ln - k * M2, b = l2 % M, c = l2 / M;
      const int s32 = (int)s, sxy = s32 / a.nx;
      const int sx = s32 - sxy * a.nx, sy = sxy % a.ny, sz = sxy / a.ny;
      int dy, iy, dz, iz;
      fdm_sub_node_g(b, n, no, &dy, &iy);
      fdm_sub_node_g(c, n, no, &dz, &iz);
      const int64_t row = a.nx * (gw(sy + dy, a.ny) + (int64_t)a.ny * gw(sz + dz, a.nz));
      const int loc = n * (iy + n * iz);
      const int64_t ol = (gw(sx - 1, a.nx) + row) * n3 + loc + (n - no);
      const int64_t oc = (sx + row) * n3 + loc - no;
      const int64_t orr = (gw(sx + 1, a.nx) + row) * n3 + loc - (no + n);
      T x[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = a.r[(t < no ? ol : (t < no + n ? oc : orr)) + t];
      T* tile = (kSmemTile ? sTile + k * M3 : a.corr + s * (int64_t)M3) + M * l2;
      gfwd<T, M>(x, sTab + k * TV, tile, 1);
    }
    __syncthreads();
    // pass 2: forward along y
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int k = ln / M2;
      const int64_t s = s0 + k;
      if (s >= a.Ne) continue;
      const int l2 = ln - k * M2;
      T* line = (kSmemTile ? sTile + k * M3 : a.corr + s * (int64_t)M3) + (l2 % M) + M2 * (l2 / M);
      T x[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = line[t * M];
      gfwd<T, M>(x, sTab + k * TV + 2 * MR, line, M);
    }
    __syncthreads();
    // pass 3: forward along z, divide by lam_x + lam_y + lam_z, backward along z
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int k = ln / M2;
      const int64_t s = s0 + k;
      if (s >= a.Ne) continue;
      const int l2 = ln - k * M2;
      const T* tb = sTab + k * TV;
      const T* lam = tb + 6 * MR;
      const T lxy = lam[l2 % M] + lam[M + l2 / M];
      T* line = (kSmemTile ? sTile + k * M3 : a.corr + s * (int64_t)M3) + l2;
      T x[M], y[M];
#pragma unroll
      for (int t = 0; t < M; ++t) x[t] = line[t * M2];
      gfwd_reg<T, M>(x, tb + 4 * MR, y);
#pragma unroll
      for (int p = 0; p < M; ++p) y[p] = y[p] / (lxy + lam[2 * M + p]);
      gbwd<T, M>(y, tb + 5 * MR, line, M2);
    }
    __syncthreads();
    // pass 4: backward along y
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int k = ln / M2;
      const int64_t s = s0 + k;
      if (s >= a.Ne) continue;
      const int l2 = ln - k * M2;
      T* line = (kSmemTile ? sTile + k * M3 : a.corr + s * (int64_t)M3) + (l2 % M) + M2 * (l2 / M);
      T v[M];
#pragma unroll
      for (int t = 0; t < M; ++t) v[t] = line[t * M];
      gbwd<T, M>(v, sTab + k * TV + 3 * MR, line, M);
    }
    __syncthreads();
    // pass 5: backward along x (weights folded into SW), into the correction buffer
    for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
      const int k = ln / M2;
      const int64_t s = s0 + k;
      if (s >= a.Ne) continue;
      const int l2 = ln - k * M2;
      const T* line = (kSmemTile ? sTile + k * M3 : a.corr + s * (int64_t)M3) + M * l2;
      T v[M];
#pragma unroll
      for (int t = 0; t < M; ++t) v[t] = line[t];
      gbwd<T, M>(v, sTab + k * TV + MR, a.corr + s * (int64_t)M3 + M * l2, 1);
    }
    __syncthreads();
  }
}

template <typename T, int M>
cudaError_t launch_gfdm_m(const mg_ctx* c, int l, const T* r) {
  const LevelInfo& lv = c->lev[l];
  GFdmMArgs<T> a;
  a.tab = gtab<T>(c);
  a.r = r;
  a.corr = static_cast<T*>(c->ws.corr);
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.n = lv.n;
  a.no = lv.no[0];
  for (int d = 0; d < 3; ++d) {
    a.S[d] = lv.t[d].gS;
    a.SW[d] = lv.t[d].gSW;
    a.lam[d] = lv.t[d].glam;
  }
  // several subdomains per block below m = 11; fewer on small meshes so that
  // the blocks still fill the SMs
  constexpr int spb_max = GShape<T, M>::spb;
  a.spb = (int)std::max<int64_t>(1, std::min<int64_t>(spb_max, (c->Ne + 2 * 152 - 1) / (2 * 152)));
  const size_t smem = GShape<T, M>::smem;
  static std::atomic<size_t> smem_set{48 * 1024};
  cudaError_t e = allow_smem((const void*)k_gfdm_m<T, M>, smem, smem_set);
  if (e != cudaSuccess) return e;
  int threads = a.spb * M * M;
  threads = threads > 256 ? 256 : (threads + 31) / 32 * 32;
  const int64_t groups = (c->Ne + a.spb - 1) / a.spb;
  const int blocks = (int)std::min<int64_t>(groups, 152 * 8);
  launch_pdl(k_gfdm_m<T, M>, blocks, threads, smem, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_gfdm_fixed(const mg_ctx* c, int l, const T* r) {
  const LevelInfo& lv = c->lev[l];
  if (lv.m[0] != lv.m[1] || lv.m[0] != lv.m[2]) return cudaErrorNotSupported;
  switch (lv.m[0]) {
#define MGDG_GCASE(M) case M: return launch_gfdm_m<T, M>(c, l, r);
    MGDG_GCASE(3) MGDG_GCASE(5) MGDG_GCASE(7) MGDG_GCASE(9) MGDG_GCASE(11) MGDG_GCASE(13) MGDG_GCASE(15)
    MGDG_GCASE(17) MGDG_GCASE(19) MGDG_GCASE(21) MGDG_GCASE(23) MGDG_GCASE(25)
#undef MGDG_GCASE
    default: return cudaErrorNotSupported;
  }
}

template cudaError_t launch_gfdm_fixed<double>(const mg_ctx*, int, const double*);
template cudaError_t launch_gfdm_fixed<float>(const mg_ctx*, int, const float*);

}  // namespace mgdg
