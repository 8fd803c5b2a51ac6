// Sum-factorised SIPG operator (Section 2, Eq. A) in FP32 or double-float
// arithmetic with shared-memory element blocks and the 1D coefficients in
// the kernel's parameter space.  (In FP64 this form was measured slower than
// the plain kernel, 248 vs 230 us on the 16^3, P = 8 level: the FP64 pipe,
// not the coefficient loads, bounds it there, so FP64 keeps the plain kernel.)
//
// The plain operator kernel (sipg_kernels.cuh) makes three passes over an
// element in global memory: every pass reads its lines with a stride and
// reads and rewrites the output vector, and every multiply-add loads its
// coefficient, so it waits on its loads.  Here a block takes EPB consecutive
// elements: their blocks of u are loaded once with coalesced loads into
// shared memory, the x, y and z line products run from there and accumulate
// in a shared output block, and the
// last (z) pass applies the mass and forms f - A u with coalesced loads of f
// and stores of the result.  Only the face terms read the neighbour lines
// from global memory (L2).  The even/odd line matrices, face vectors, rows of
// the differentiation matrix and the 1D masses (at most 4.2 KB at n = 17 in
// double-float) travel as one __grid_constant__ parameter, so with the
// compile-time order every coefficient is an immediate constant-bank operand.
// The arithmetic is that of line_apply_n (the same even/odd form, face terms,
// accumulation (Acc) and order of the three directions); the mass of a node
// is formed as the product of the three 1D masses.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "mg_internal.h"

namespace mgdg {
namespace {

template <typename T, int N>
struct SipgCShape {
  static constexpr int ne = (N + 1) / 2, no = N / 2, noo = no > 0 ? no : 1;
  static constexpr int n2 = N * N, n3 = n2 * N;
  static constexpr int epb = n2 >= 256 ? 1 : 256 / n2;  // elements per block
  static constexpr int threads = (epb * n2 + 31) / 32 * 32;
  static constexpr size_t smem = sizeof(T) * 2 * (size_t)epb * n3;
};

template <typename T, int N>
struct SipgCArgs {
  using Sh = SipgCShape<T, N>;
  const T* u;
  const T* f;
  T* out;
  int64_t Ne;
  int nx, ny, nz, residual;
  T ce[3][Sh::ne * Sh::ne];    // even half of M_d^{-1} L_ee
  T co[3][Sh::noo * Sh::noo];  // odd half
  T fe[3][Sh::ne], fo[3][Sh::noo];  // face vectors of the even / odd halves
  T mu[3], g2[3];              // face scalars mu / m_0 and g / (2 m_0)
  T d0[N], dp[N];              // first and last row of the reference differentiation matrix
  T mass[3][N];                // 1D masses (h_d / 2) w
};

template <typename T>
__device__ __forceinline__ T sc_load(const T* p) {
  return *p;
}
template <>
__device__ __forceinline__ float sc_load<float>(const float* p) {
  return __ldg(p);
}

__device__ __forceinline__ int sc_wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// One line of direction D: the own line from shared memory (stride st), the
// face terms from the neighbours' lines in global memory, outputs combined
// into the shared output block (D = 0: store, 1: add) or, for D = 2, into
// out = residual ? f - M (acc + v) : M (acc + v) in global memory.
// SPLIT (the direction-split kernel): su is the line in global memory, the
// x and y contributions accumulate in out itself (so == out for D < 2; for
// D = 2 they are read back from out).
template <typename T, int N, int D, bool SPLIT = false>
__device__ __forceinline__ void line_c(const SipgCArgs<T, N>& a, const T* __restrict__ su, T* so,
                                       const T* __restrict__ uL, const T* __restrict__ uR, int st,
                                       T* out, const T* __restrict__ fl, T mpq) {
  constexpr int P = N - 1, ne = (N + 1) / 2, no = N / 2;
  T ev[ne], od[no > 0 ? no : 1];
#pragma unroll
  for (int t = 0; t < no; ++t) {
    const T xa = su[t * st], xb = su[(P - t) * st];
    ev[t] = xa + xb;
    od[t] = xa - xb;
  }
  if (N & 1) ev[ne - 1] = su[no * st];
  const T av = sc_load(uL + P * st), cv = sc_load(uR);
  Acc<T> ba, da;
  ba.init(a.dp[0], sc_load(uL));
  da.init(a.d0[0], cv);
#pragma unroll
  for (int t = 1; t < N; ++t) {
    ba.add(a.dp[t], sc_load(uL + t * st));
    da.add(a.d0[t], sc_load(uR + t * st));
  }
  const T b = ba.get(), dd = da.get();
  const T s = av + cv, tm = av - cv;
  const T lo = a.g2[D] * b - a.mu[D] * av;
  const T hi = -(a.mu[D] * cv + a.g2[D] * dd);
  // double-float at n = 33: the fully unrolled outputs overflow the
  // instruction cache (the kernel stalled on instruction fetch), so one output
  // per trip, its products unrolled, the coefficients indexed by the trip
  // (1.66 vs 2.59 ms per P = 32 solve; in FP32 rolling measured slower)
  constexpr int kUnroll = (std::is_same<T, df64>::value && N >= 33) ? 1 : ne;
#pragma unroll kUnroll
  for (int i = 0; i < ne; ++i) {
    Acc<T> ea;
    ea.init(a.fe[D][i], s);
#pragma unroll
    for (int t = 0; t < ne; ++t) ea.add(a.ce[D][i * ne + t], ev[t]);
    const T E = ea.get();
    T v0, v1;
    if (i < no) {
      Acc<T> oa;
      oa.init(a.fo[D][i], tm);
#pragma unroll
      for (int t = 0; t < no; ++t) oa.add(a.co[D][i * no + t], od[t]);
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
    if (D == 0) {
      so[i * st] = v0;
      if (i1 != i) so[i1 * st] = v1;
    } else if (D == 1) {
      so[i * st] += v0;
      if (i1 != i) so[i1 * st] += v1;
    } else {
      const T* acc = SPLIT ? out : so;
      const T w0 = mpq * a.mass[2][i] * (acc[i * st] + v0);
      const T w1 = mpq * a.mass[2][i1] * (acc[i1 * st] + v1);
      out[i * st] = a.residual ? fl[i * st] - w0 : w0;
      if (i1 != i) out[i1 * st] = a.residual ? fl[i1 * st] - w1 : w1;
    }
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(SipgCShape<T, N>::threads) k_sipg_c(const __grid_constant__ SipgCArgs<T, N> a) {
  pdl_entry();
  using Sh = SipgCShape<T, N>;
  constexpr int n2 = Sh::n2, n3 = Sh::n3, EPB = Sh::epb;
  extern __shared__ __align__(16) unsigned char sc_raw[];
  T* sU = reinterpret_cast<T*>(sc_raw);  // EPB element blocks of u
  T* sO = sU + EPB * n3;                 // EPB output blocks (x and y contributions)
  const int tid = threadIdx.x, nt = blockDim.x;
  const int g = tid / n2, l2 = tid - g * n2, p = l2 % N, q = l2 / N;
  for (int64_t e0 = (int64_t)blockIdx.x * EPB; e0 < a.Ne; e0 += (int64_t)gridDim.x * EPB) {
    const int cnt = (int)(a.Ne - e0 < EPB ? a.Ne - e0 : EPB);
    const T* ub = a.u + e0 * n3;
    for (int i = tid; i < cnt * n3; i += nt) sU[i] = ub[i];
    __syncthreads();
    const bool act = g < cnt;
    int ex = 0, ey = 0, ez = 0;
    if (act) {
      const int e32 = (int)(e0 + g), exy = e32 / a.nx;  // element indices fit in 32 bits
      ex = e32 - exy * a.nx;
      ey = exy % a.ny;
      ez = exy / a.ny;
    }
    const T* su = sU + g * n3;
    T* so = sO + g * n3;
    if (act) {  // x lines (p, q) = (j, k)
      const int base = N * (p + N * q);
      const int64_t row = (int64_t)a.nx * (ey + (int64_t)a.ny * ez);
      line_c<T, N, 0>(a, su + base, so + base, a.u + (sc_wrap(ex - 1, a.nx) + row) * n3 + base,
                      a.u + (sc_wrap(ex + 1, a.nx) + row) * n3 + base, 1, nullptr, nullptr, T(0.f));
    }
    __syncthreads();
    if (act) {  // y lines (p, q) = (i, k)
      const int base = p + n2 * q;
      const int64_t eL = ex + a.nx * (sc_wrap(ey - 1, a.ny) + (int64_t)a.ny * ez);
      const int64_t eR = ex + a.nx * (sc_wrap(ey + 1, a.ny) + (int64_t)a.ny * ez);
      line_c<T, N, 1>(a, su + base, so + base, a.u + eL * n3 + base, a.u + eR * n3 + base, N, nullptr, nullptr,
                      T(0.f));
    }
    __syncthreads();
    if (act) {  // z lines (p, q) = (i, j): mass, residual, coalesced stores
      const int base = p + N * q;
      const int64_t exy = ex + (int64_t)a.nx * ey, plane = (int64_t)a.nx * a.ny;
      const int64_t eL = exy + plane * sc_wrap(ez - 1, a.nz), eR = exy + plane * sc_wrap(ez + 1, a.nz);
      const int64_t off = (e0 + g) * n3 + base;
      line_c<T, N, 2>(a, su + base, so + base, a.u + eL * n3 + base, a.u + eR * n3 + base, n2, a.out + off,
                      a.residual ? a.f + off : nullptr, a.mass[0][p] * a.mass[1][q]);
    }
    __syncthreads();
  }
}

// Direction-split form for meshes with few elements (too few blocks of
// element blocks to fill the SMs; n = 33 always, whose element block does not
// fit shared memory): three launches, one thread per line of direction D of
// every element, the own line read from global memory, the contributions of
// x and y accumulated in the output vector and the z launch applying the
// mass and forming f - A u there.  Same arithmetic as k_sipg_c, with the
// coefficients in the parameter space.
template <typename T, int N, int D>
__global__ void __launch_bounds__(256) k_sipg_cd(const __grid_constant__ SipgCArgs<T, N> a) {
  pdl_entry();
  constexpr int n2 = N * N, n3 = n2 * N;
  const int64_t gl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t e = gl / n2;
  if (e >= a.Ne) return;
  const int l2 = (int)(gl - e * n2), p = l2 % N, q = l2 / N;
  const int e32 = (int)e, exy = e32 / a.nx;  // element indices fit in 32 bits
  const int ex = e32 - exy * a.nx, ey = exy % a.ny, ez = exy / a.ny;
  if (D == 0) {  // x lines (p, q) = (j, k)
    const int base = N * (p + N * q);
    const int64_t row = (int64_t)a.nx * (ey + (int64_t)a.ny * ez);
    T* o = a.out + e * n3 + base;
    line_c<T, N, 0, true>(a, a.u + e * n3 + base, o, a.u + (sc_wrap(ex - 1, a.nx) + row) * n3 + base,
                          a.u + (sc_wrap(ex + 1, a.nx) + row) * n3 + base, 1, nullptr, nullptr, T(0.f));
  } else if (D == 1) {  // y lines (p, q) = (i, k)
    const int base = p + n2 * q;
    const int64_t eL = ex + a.nx * (sc_wrap(ey - 1, a.ny) + (int64_t)a.ny * ez);
    const int64_t eR = ex + a.nx * (sc_wrap(ey + 1, a.ny) + (int64_t)a.ny * ez);
    T* o = a.out + e * n3 + base;
    line_c<T, N, 1, true>(a, a.u + e * n3 + base, o, a.u + eL * n3 + base, a.u + eR * n3 + base, N, nullptr,
                          nullptr, T(0.f));
  } else {  // z lines (p, q) = (i, j): mass, residual
    const int base = p + N * q;
    const int64_t exy2 = ex + (int64_t)a.nx * ey, plane = (int64_t)a.nx * a.ny;
    const int64_t eL = exy2 + plane * sc_wrap(ez - 1, a.nz), eR = exy2 + plane * sc_wrap(ez + 1, a.nz);
    const int64_t off = e * n3 + base;
    line_c<T, N, 2, true>(a, a.u + off, nullptr, a.u + eL * n3 + base, a.u + eR * n3 + base, n2, a.out + off,
                          a.residual ? a.f + off : nullptr, a.mass[0][p] * a.mass[1][q]);
  }
}

template <typename T>
const std::vector<T>& host_tables(const mg_ctx* c);
template <>
const std::vector<float>& host_tables<float>(const mg_ctx* c) { return c->tab32_host; }
template <>
const std::vector<df64>& host_tables<df64>(const mg_ctx* c) { return c->tabdf_host; }

template <typename T, int N>
void fill_sipg_c_args(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual, SipgCArgs<T, N>& a) {
  using Sh = SipgCShape<T, N>;
  constexpr int ne = Sh::ne, no = Sh::no;
  static_assert(sizeof(SipgCArgs<T, N>) <= 32000, "parameter block too large");
  const LevelInfo& lv = c->lev[l];
  const T* tab = host_tables<T>(c).data();
  a.u = u;
  a.f = f;
  a.out = out;
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.residual = residual;
  for (int d = 0; d < 3; ++d) {
    const DirTables& t = lv.t[d];
    for (int i = 0; i < ne * ne; ++i) a.ce[d][i] = tab[t.ce + i];
    for (int i = 0; i < no * no; ++i) a.co[d][i] = tab[t.co + i];
    for (int i = 0; i < ne; ++i) a.fe[d][i] = tab[t.fe + i];
    for (int i = 0; i < no; ++i) a.fo[d][i] = tab[t.fo + i];
    a.mu[d] = tab[t.fsc];
    a.g2[d] = tab[t.fsc + 1];
    for (int i = 0; i < N; ++i) a.mass[d][i] = tab[t.mass + i];
  }
  for (int i = 0; i < N; ++i) {
    a.d0[i] = tab[lv.t[0].d0 + i];
    a.dp[i] = tab[lv.t[0].dp + i];
  }
}

template <typename T, int N>
cudaError_t launch_sipg_c_n(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual) {
  using Sh = SipgCShape<T, N>;
  SipgCArgs<T, N> a;
  fill_sipg_c_args<T, N>(c, l, u, f, out, residual, a);
  if (Sh::smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_sipg_c<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    if (e != cudaSuccess) return e;
  }
  static std::atomic<int> per_sm_cached{0};  // resident blocks per SM, queried once per type and order
  int per_sm = per_sm_cached.load();
  if (per_sm == 0) {
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sipg_c<T, N>, Sh::threads, Sh::smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    per_sm_cached.store(per_sm);
  }
  const int64_t groups = (c->Ne + Sh::epb - 1) / Sh::epb;
  const int blocks = (int)std::min<int64_t>(groups, 152LL * per_sm);
  launch_pdl(k_sipg_c<T, N>, blocks, Sh::threads, Sh::smem, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t launch_sipg_cd_n(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual) {
  SipgCArgs<T, N> a;
  fill_sipg_c_args<T, N>(c, l, u, f, out, residual, a);
  const int64_t blocks = (c->Ne * (int64_t)(N * N) + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorNotSupported;
  launch_pdl(k_sipg_cd<T, N, 0>, (int)blocks, 256, 0, c->stream, a);
  launch_pdl(k_sipg_cd<T, N, 1>, (int)blocks, 256, 0, c->stream, a);
  launch_pdl(k_sipg_cd<T, N, 2>, (int)blocks, 256, 0, c->stream, a);
  c->nlaunch += 3;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sipg_c_t(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual) {
  if (host_tables<T>(c).empty()) return cudaErrorNotSupported;
  const int n = c->lev[l].n;
  const int epb = n * n >= 256 ? 1 : 256 / (n * n);
  if (n == 33) return launch_sipg_cd_n<T, 33>(c, l, u, f, out, residual);
  if ((c->Ne + epb - 1) / epb < 152) {
    // too few element blocks to fill the SMs: the direction-split form (high
    // orders; the low ones keep the plain direction-split kernel)
    if (n == 17) return launch_sipg_cd_n<T, 17>(c, l, u, f, out, residual);
    if (n == 9) return launch_sipg_cd_n<T, 9>(c, l, u, f, out, residual);
    return cudaErrorNotSupported;
  }
  switch (n) {
    case 3: return launch_sipg_c_n<T, 3>(c, l, u, f, out, residual);
    case 5: return launch_sipg_c_n<T, 5>(c, l, u, f, out, residual);
    case 9: return launch_sipg_c_n<T, 9>(c, l, u, f, out, residual);
    case 17: return launch_sipg_c_n<T, 17>(c, l, u, f, out, residual);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t launch_sipg_c(const mg_ctx* c, int l, const float* u, const float* f, float* out, int residual) {
  return launch_sipg_c_t<float>(c, l, u, f, out, residual);
}

cudaError_t launch_sipg_c(const mg_ctx* c, int l, const df64* u, const df64* f, df64* out, int residual) {
  return launch_sipg_c_t<df64>(c, l, u, f, out, residual);
}

}  // namespace mgdg
