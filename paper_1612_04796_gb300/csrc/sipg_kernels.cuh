// Sum-factorised SIPG operator (Section 2, Eq. A):
//   A = Mz(x)My(x)Lx + Mz(x)Ly(x)Mx + Lz(x)My(x)Mx = M (I(x)I(x)Cx + I(x)Cy(x)I + Cz(x)I(x)I),
// with M = Mz(x)My(x)Mx the diagonal mass and C_d = M_d^{-1} L_d, applied
// element by element.  Row block e of the 1D matrix L is
//   L_ee u_e + L_e,e-1 u_e-1 + L_e,e+1 u_e+1,
// where L_ee = (2/h) D^T W D plus the self terms of both faces and the
// neighbour couplings are rank-2 face terms (standard SIPG reading of Eq. ip):
//   (L_e,e-1 u_e-1)_i = delta_i0 (-mu a + g/2 b) - g/2 D0_i a,
//        a = u_e-1 at its node P, b = (D u_e-1) at its node P,
//   (L_e,e+1 u_e+1)_i = delta_iP (-mu c - g/2 d) + g/2 DP_i c,
//        c = u_e+1 at its node 0, d = (D u_e+1) at its node 0,
// with g = 2/h and D0 / DP the first / last row of the reference
// differentiation matrix.
//
// L_ee and M_d are symmetric under reflection of the element (i -> P-i) and
// DP_i = -D0_{P-i}, so every 1D line product is evaluated in even/odd form:
// e_t = u_t + u_{P-t}, o_t = u_t - u_{P-t}; two half-size products; the face
// rank-1 terms fold into the even part (with a + c) and the odd part (with
// a - c).  One thread per 1D line; the three directions are three passes over
// the element, accumulated in the output vector; the last pass applies the
// mass and forms f - A u.  The kernels are templates on the arithmetic type:
// FP64, FP32 (the multigrid of the mixed solve) or double-float pairs
// (df64.cuh; the outer operator of the mixed solve on request).  Included by
// sipg_f64.cu, sipg_f32.cu and sipg_df64.cu, one arithmetic type each.
#pragma once

#include "mg_internal.h"

namespace mgdg {
namespace {

constexpr int kMaxHalf = kMaxN / 2 + 1;

template <typename T>
struct OpArgs {
  const T* tab;
  const T* u;
  const T* f;
  T* out;
  int64_t Ne;
  int nx, ny, nz, n, residual, epb;
  int64_t ce[3], co[3], fe[3], fo[3], fsc[3], d0, dp, mass3;
};

// One direction of one line.  ue / uL / uR: the line in the element and in
// its left / right neighbour (same stride st); o: the output line.
// mode 0: o = C u; 1: o += C u; 2: o = residual ? f - M (o + C u) : M (o + C u).
template <typename T>
__device__ __forceinline__ void line_apply(const OpArgs<T>& a, int d, const T* __restrict__ ue,
                                           const T* __restrict__ uL, const T* __restrict__ uR, int st, T* o,
                                           const T* __restrict__ fl, const T* __restrict__ m3, int m3st, int mode) {
  const int n = a.n, P = n - 1, ne = (n + 1) / 2, no = n / 2;
  const T* __restrict__ ce = a.tab + a.ce[d];
  const T* __restrict__ co = a.tab + a.co[d];
  const T* __restrict__ fe = a.tab + a.fe[d];
  const T* __restrict__ fo = a.tab + a.fo[d];
  const T* __restrict__ D0 = a.tab + a.d0;
  const T* __restrict__ DP = a.tab + a.dp;
  const T mu_m0 = a.tab[a.fsc[d]], g2_m0 = a.tab[a.fsc[d] + 1];
  T ev[kMaxHalf], od[kMaxHalf];
  for (int t = 0; t < no; ++t) {
    const T xa = ue[t * st], xb = ue[(P - t) * st];
    ev[t] = xa + xb;
    od[t] = xa - xb;
  }
  if (n & 1) ev[no] = ue[no * st];
  const T av = uL[P * st], cv = uR[0];
  T b = 0, dd = 0;
  for (int t = 0; t < n; ++t) {
    b += DP[t] * uL[t * st];
    dd += D0[t] * uR[t * st];
  }
  const T s = av + cv, tm = av - cv;
  const T lo = g2_m0 * b - mu_m0 * av;     // extra term of output 0
  const T hi = -(mu_m0 * cv + g2_m0 * dd);  // extra term of output P
  for (int i = 0; i < ne; ++i) {
    T E = fe[i] * s;
    for (int t = 0; t < ne; ++t) E += ce[i * ne + t] * ev[t];
    T v0, v1;
    if (i < no) {
      T O = fo[i] * tm;
      for (int t = 0; t < no; ++t) O += co[i * no + t] * od[t];
      v0 = E + O;
      v1 = E - O;
    } else {
      v0 = v1 = E;
    }
    if (i == 0) {
      v0 += lo;
      v1 += hi;
    }
    const int i1 = P - i;
    if (mode == 0) {
      o[i * st] = v0;
      if (i1 != i) o[i1 * st] = v1;
    } else if (mode == 1) {
      o[i * st] += v0;
      if (i1 != i) o[i1 * st] += v1;
    } else {
      const T w0 = m3[i * m3st] * (o[i * st] + v0);
      o[i * st] = a.residual ? fl[i * st] - w0 : w0;
      if (i1 != i) {
        const T w1 = m3[i1 * m3st] * (o[i1 * st] + v1);
        o[i1 * st] = a.residual ? fl[i1 * st] - w1 : w1;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sipg(OpArgs<T> a) {
  pdl_entry();
  const int n = a.n, n2 = n * n, n3 = n2 * n, P = n - 1;
  const int lines = a.epb * n2;
  const T* m3 = a.tab + a.mass3;
  for (int64_t e0 = (int64_t)blockIdx.x * a.epb; e0 < a.Ne; e0 += (int64_t)gridDim.x * a.epb) {
    for (int dir = 0; dir < 3; ++dir) {
      for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
        const int64_t e = e0 + ln / n2;
        if (e >= a.Ne) continue;
        const int l2 = ln % n2, p = l2 % n, q = l2 / n;
        const int e32 = (int)e, exy = e32 / a.nx;  // element indices fit in 32 bits
        const int ex = e32 - exy * a.nx, ey = exy % a.ny, ez = exy / a.ny;
        int64_t eL, eR;
        int base, st;
        if (dir == 0) {
          eL = (ex == 0 ? a.nx - 1 : ex - 1) + a.nx * (ey + (int64_t)a.ny * ez);
          eR = (ex == a.nx - 1 ? 0 : ex + 1) + a.nx * (ey + (int64_t)a.ny * ez);
          base = n * (p + n * q);
          st = 1;
        } else if (dir == 1) {
          eL = ex + a.nx * ((ey == 0 ? a.ny - 1 : ey - 1) + (int64_t)a.ny * ez);
          eR = ex + a.nx * ((ey == a.ny - 1 ? 0 : ey + 1) + (int64_t)a.ny * ez);
          base = p + n2 * q;
          st = n;
        } else {
          eL = ex + a.nx * (ey + (int64_t)a.ny * (ez == 0 ? a.nz - 1 : ez - 1));
          eR = ex + a.nx * (ey + (int64_t)a.ny * (ez == a.nz - 1 ? 0 : ez + 1));
          base = p + n * q;
          st = n2;
        }
        const int64_t off = e * n3 + base;
        line_apply<T>(a, dir, a.u + off, a.u + eL * n3 + base, a.u + eR * n3 + base, st, a.out + off,
                      a.residual ? a.f + off : nullptr, m3 + base, st, dir);
      }
      __syncthreads();
    }
  }
  (void)P;
}

// Compile-time-size version of line_apply / k_sipg (lines in registers).
// NP > 1: the line's output pairs (i, P - i) are shared by NP threads, thread
// `part` taking i = part, part + NP, ...; each reads the whole line.
template <typename T, int N, int NP = 1>
__device__ __forceinline__ void line_apply_n(const OpArgs<T>& a, int d, const T* __restrict__ ue,
                                             const T* __restrict__ uL, const T* __restrict__ uR, int st, T* o,
                                             const T* __restrict__ fl, const T* __restrict__ m3, int mode,
                                             int part = 0) {
  constexpr int P = N - 1, ne = (N + 1) / 2, no = N / 2;
  const T* __restrict__ ce = a.tab + a.ce[d];
  const T* __restrict__ co = a.tab + a.co[d];
  const T* __restrict__ fe = a.tab + a.fe[d];
  const T* __restrict__ fo = a.tab + a.fo[d];
  const T* __restrict__ D0 = a.tab + a.d0;
  const T* __restrict__ DP = a.tab + a.dp;
  const T mu_m0 = a.tab[a.fsc[d]], g2_m0 = a.tab[a.fsc[d] + 1];
  T ev[ne], od[no > 0 ? no : 1];
#pragma unroll
  for (int t = 0; t < no; ++t) {
    const T xa = ue[t * st], xb = ue[(P - t) * st];
    ev[t] = xa + xb;
    od[t] = xa - xb;
  }
  if (N & 1) ev[ne - 1] = ue[no * st];
  const T av = uL[P * st], cv = uR[0];
  Acc<T> ba, da;
  ba.init(DP[0], uL[0]);
  da.init(D0[0], uR[0]);
#pragma unroll
  for (int t = 1; t < N; ++t) {
    ba.add(DP[t], uL[t * st]);
    da.add(D0[t], uR[t * st]);
  }
  const T b = ba.get(), dd = da.get();
  const T s = av + cv, tm = av - cv;
  const T lo = g2_m0 * b - mu_m0 * av;
  const T hi = -(mu_m0 * cv + g2_m0 * dd);
#pragma unroll
  for (int ii = 0; ii < (ne + NP - 1) / NP; ++ii) {
    const int i = NP == 1 ? ii : part + ii * NP;
    if (NP > 1 && i >= ne) break;
    Acc<T> ea;
    ea.init(fe[i], s);
#pragma unroll
    for (int t = 0; t < ne; ++t) ea.add(ce[i * ne + t], ev[t]);
    const T E = ea.get();
    T v0, v1;
    if (i < no) {
      Acc<T> oa;
      oa.init(fo[i], tm);
#pragma unroll
      for (int t = 0; t < no; ++t) oa.add(co[i * no + t], od[t]);
      const T O = oa.get();
      v0 = E + O;
      v1 = E - O;
    } else {
      v0 = v1 = E;
    }
    if (i == 0) {
      v0 += lo;
      v1 += hi;
    }
    const int i1 = P - i;
    if (mode == 0) {
      o[i * st] = v0;
      if (i1 != i) o[i1 * st] = v1;
    } else if (mode == 1) {
      o[i * st] += v0;
      if (i1 != i) o[i1 * st] += v1;
    } else {
      const T w0 = m3[i * st] * (o[i * st] + v0);
      o[i * st] = a.residual ? fl[i * st] - w0 : w0;
      if (i1 != i) {
        const T w1 = m3[i1 * st] * (o[i1 * st] + v1);
        o[i1 * st] = a.residual ? fl[i1 * st] - w1 : w1;
      }
    }
  }
}

template <typename T, int N>
__device__ __forceinline__ void sipg_n_body(BlockIdx bi, OpArgs<T> a) {
  constexpr int n2 = N * N, n3 = n2 * N;
  const int lines = a.epb * n2;
  const T* m3 = a.tab + a.mass3;
  for (int64_t e0 = (int64_t)bi.b * a.epb; e0 < a.Ne; e0 += (int64_t)bi.g * a.epb) {
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      for (int ln = threadIdx.x; ln < lines; ln += blockDim.x) {
        const int64_t e = e0 + ln / n2;
        if (e >= a.Ne) continue;
        const int l2 = ln % n2, p = l2 % N, q = l2 / N;
        const int e32 = (int)e, exy = e32 / a.nx;  // element indices fit in 32 bits
        const int ex = e32 - exy * a.nx, ey = exy % a.ny, ez = exy / a.ny;
        int64_t eL, eR;
        int base, st;
        if (dir == 0) {
          eL = (ex == 0 ? a.nx - 1 : ex - 1) + a.nx * (ey + (int64_t)a.ny * ez);
          eR = (ex == a.nx - 1 ? 0 : ex + 1) + a.nx * (ey + (int64_t)a.ny * ez);
          base = N * (p + N * q);
          st = 1;
        } else if (dir == 1) {
          eL = ex + a.nx * ((ey == 0 ? a.ny - 1 : ey - 1) + (int64_t)a.ny * ez);
          eR = ex + a.nx * ((ey == a.ny - 1 ? 0 : ey + 1) + (int64_t)a.ny * ez);
          base = p + n2 * q;
          st = N;
        } else {
          eL = ex + a.nx * (ey + (int64_t)a.ny * (ez == 0 ? a.nz - 1 : ez - 1));
          eR = ex + a.nx * (ey + (int64_t)a.ny * (ez == a.nz - 1 ? 0 : ez + 1));
          base = p + N * q;
          st = n2;
        }
        const int64_t off = e * n3 + base;
        line_apply_n<T, N>(a, dir, a.u + off, a.u + eL * n3 + base, a.u + eR * n3 + base, st, a.out + off,
                           a.residual ? a.f + off : nullptr, m3 + base, dir);
      }
      __syncthreads();
    }
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_sipg_n(OpArgs<T> a) {
  pdl_entry();
  sipg_n_body<T, N>(plain_block(), a);
}

// Direction-split variant for meshes with few elements: one launch per
// direction, each element's lines (times NP threads per line) spread over
// `chunks` blocks.
template <typename T, int N, int NP>
__device__ __forceinline__ void sipg_dir_body(BlockIdx blk, OpArgs<T> a, int dir, int chunks) {
  constexpr int n2 = N * N, n3 = n2 * N;
  const T* m3 = a.tab + a.mass3;
  const int64_t nblk = a.Ne * chunks;
  for (int64_t bi = blk.b; bi < nblk; bi += blk.g) {
    const int64_t e = bi / chunks;
    const int lt = (int)(bi % chunks) * blockDim.x + threadIdx.x;
    if (lt >= n2 * NP) continue;
    const int ln = lt / NP, part = lt - ln * NP;
    const int p = ln % N, q = ln / N;
    const int e32 = (int)e, exy = e32 / a.nx;  // element indices fit in 32 bits
    const int ex = e32 - exy * a.nx, ey = exy % a.ny, ez = exy / a.ny;
    int64_t eL, eR;
    int base, st;
    if (dir == 0) {
      eL = (ex == 0 ? a.nx - 1 : ex - 1) + a.nx * (ey + (int64_t)a.ny * ez);
      eR = (ex == a.nx - 1 ? 0 : ex + 1) + a.nx * (ey + (int64_t)a.ny * ez);
      base = N * (p + N * q);
      st = 1;
    } else if (dir == 1) {
      eL = ex + a.nx * ((ey == 0 ? a.ny - 1 : ey - 1) + (int64_t)a.ny * ez);
      eR = ex + a.nx * ((ey == a.ny - 1 ? 0 : ey + 1) + (int64_t)a.ny * ez);
      base = p + n2 * q;
      st = N;
    } else {
      eL = ex + a.nx * (ey + (int64_t)a.ny * (ez == 0 ? a.nz - 1 : ez - 1));
      eR = ex + a.nx * (ey + (int64_t)a.ny * (ez == a.nz - 1 ? 0 : ez + 1));
      base = p + N * q;
      st = n2;
    }
    const int64_t off = e * n3 + base;
    line_apply_n<T, N, NP>(a, dir, a.u + off, a.u + eL * n3 + base, a.u + eR * n3 + base, st, a.out + off,
                           a.residual ? a.f + off : nullptr, m3 + base, dir, part);
  }
}

template <typename T, int N, int NP>
__global__ void __launch_bounds__(256) k_sipg_dir(OpArgs<T> a, int dir, int chunks) {
  pdl_entry();
  sipg_dir_body<T, N, NP>(plain_block(), a, dir, chunks);
}

// The three direction launches of the direction-split operator, NP threads per line.
template <typename T, int N, int NP>
cudaError_t launch_sipg_dir(const mg_ctx* c, OpArgs<T>& a) {
  constexpr int n2 = N * N;
  const int chunks = (n2 * NP + 255) / 256;
  const int threads = ((n2 * NP + chunks - 1) / chunks + 31) / 32 * 32;
  const int64_t nblk = c->Ne * chunks;
  const int blocks = (int)(nblk < 152 * 16 ? nblk : 152 * 16);
  for (int dir = 0; dir < 3; ++dir) {
    launch_pdl<kTwinType<T> ? &sipg_dir_body<T, N, NP> : nullptr>(k_sipg_dir<T, N, NP>, blocks, threads, 0,
                                                                  c->stream, a, dir, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  c->nlaunch += 3;
  return cudaSuccess;
}

template <typename T, int N>
cudaError_t launch_sipg_n(const mg_ctx* c, OpArgs<T>& a) {
  constexpr int n2 = N * N;
  // lines per element and direction spread evenly over <= 256 threads
  const int iters = (n2 + 255) / 256;
  if (iters > 1 || c->Ne < 2 * 152) {
    // The long lines of high orders are shared by 4 threads on meshes of few
    // elements (4 times the parallelism).  Every sharing thread repeats the
    // line's even/odd and face sums, so with enough lines (the 48x8x8, P = 16
    // mesh has 888k per direction) each line gets one thread.
    const bool share = N >= 17 && c->Ne * (int64_t)n2 < 152 * 512;
    const int np = share ? 4 : 1;
    const int chunks = (n2 * np + 255) / 256;
    if (c->Ne * chunks < 4 * 152 || iters > 1)
      return share ? launch_sipg_dir<T, N, (N >= 17 ? 4 : 1)>(c, a) : launch_sipg_dir<T, N, 1>(c, a);
  }
  a.epb = n2 >= 128 ? 1 : 128 / n2;
  int threads = a.epb * n2;
  threads = (threads + 31) / 32 * 32;
  if (threads > 256) threads = 256;
  int64_t groups = (c->Ne + a.epb - 1) / a.epb;
  int64_t blocks = groups < 152 * 16 ? groups : 152 * 16;
  launch_pdl<kTwinType<T> ? &sipg_n_body<T, N> : nullptr>(k_sipg_n<T, N>, (int)blocks, threads, 0, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T>
const T* table_of(const mg_ctx* c);
template <>
const double* table_of<double>(const mg_ctx* c) { return c->ws.tab64; }
template <>
const float* table_of<float>(const mg_ctx* c) { return c->ws.tab32; }
template <>
const df64* table_of<df64>(const mg_ctx* c) { return c->ws.tabdf; }

}  // namespace

template <typename T>
cudaError_t launch_sipg(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual) {
  if (c->graded) return launch_gsipg<T>(c, l, u, f, out, residual);
  const LevelInfo& lv = c->lev[l];
  OpArgs<T> a;
  a.tab = table_of<T>(c);
  a.u = u;
  a.f = f;
  a.out = out;
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.n = lv.n;
  a.residual = residual;
  for (int d = 0; d < 3; ++d) {
    a.ce[d] = lv.t[d].ce;
    a.co[d] = lv.t[d].co;
    a.fe[d] = lv.t[d].fe;
    a.fo[d] = lv.t[d].fo;
    a.fsc[d] = lv.t[d].fsc;
  }
  a.d0 = lv.t[0].d0;
  a.dp = lv.t[0].dp;
  a.mass3 = lv.mass3;
  if constexpr (!std::is_same<T, double>::value) {
    // single solves (FP32, double-float): shared-memory element blocks,
    // coefficients as kernel parameters; batched solves keep the kernels
    // whose bodies have twins
    if (launch_recorder() == nullptr && !lv.sipg_plain) {
      const cudaError_t e = launch_sipg_c(c, l, u, f, out, residual);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  const int n2 = lv.n * lv.n;
  a.epb = n2 >= 128 ? 1 : 128 / n2;
  int threads = a.epb * n2;
  threads = (threads + 31) / 32 * 32;
  if (threads > 256) threads = 256;
  int64_t groups = (c->Ne + a.epb - 1) / a.epb;
  int64_t blocks = groups < 152 * 16 ? groups : 152 * 16;
  switch (lv.n) {
    case 2: return launch_sipg_n<T, 2>(c, a);
    case 3: return launch_sipg_n<T, 3>(c, a);
    case 5: return launch_sipg_n<T, 5>(c, a);
    case 9: return launch_sipg_n<T, 9>(c, a);
    case 17: return launch_sipg_n<T, 17>(c, a);
    case 33: return launch_sipg_n<T, 33>(c, a);
    default: break;
  }
  c->nlaunch += 1;
  launch_pdl(k_sipg<T>, (int)blocks, threads, 0, c->stream, a);
  return cudaGetLastError();
}

}  // namespace mgdg
