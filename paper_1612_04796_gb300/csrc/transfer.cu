// Polynomial transfers between levels (Section 3.2, Algorithm 1):
//   prolongation  u_l += I_l u_{l-1},    I_l = J (x) J (x) J per element,
//   restriction   f_{l-1} = I_l^T r_l,
// with J (n_f x n_c) the values of the order-P_{l-1} GLL Lagrange basis at the
// order-P_l GLL nodes (embedded interpolation).  Both are applied as three
// one-axis contractions (sum factorisation), one output value per thread,
// through the smoother's correction buffer as scratch (order 32), or in one
// fused kernel with shared-memory intermediates and even/odd products, a few
// elements per block pass (orders 2..16).
#include <type_traits>

#include "mg_internal.h"

namespace mgdg {
namespace {

// out[e][...o...] (+)= sum_t Mat(o, t) in[e][...t...] along `axis` of a
// per-element tensor with extents (d0, d1, d2), x fastest.
// Mat(o, t) = transpose ? J[t * ldj + o] : J[o * ldj + t].
template <typename T>
__device__ __forceinline__ void contract_axis_body(BlockIdx bi_, const T* __restrict__ in, T* __restrict__ out,
                                                   const T* __restrict__ J, int64_t Ne, int d0, int d1, int d2,
                                                   int axis, int nout, int ldj, int transpose, int accumulate) {
  int o0 = d0, o1 = d1, o2 = d2;
  if (axis == 0) o0 = nout; else if (axis == 1) o1 = nout; else o2 = nout;
  const int64_t in_sz = (int64_t)d0 * d1 * d2, out_sz = (int64_t)o0 * o1 * o2;
  const int64_t total = Ne * out_sz;
  const int nin = axis == 0 ? d0 : (axis == 1 ? d1 : d2);
  for (int64_t idx = bi_.b * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)bi_.g * blockDim.x) {
    const int64_t e = idx / out_sz;
    const int loc = (int)(idx - e * out_sz);
    const int a = loc % o0, b = (loc / o0) % o1, c = loc / (o0 * o1);
    const T* src = in + e * in_sz;
    int base, stride, o;
    if (axis == 0) { base = d0 * (b + d1 * c); stride = 1; o = a; }
    else if (axis == 1) { base = a + d0 * d1 * c; stride = d0; o = b; }
    else { base = a + d0 * b; stride = d0 * d1; o = c; }
    T acc = 0;
    for (int t = 0; t < nin; ++t) {
      const T m = transpose ? J[t * ldj + o] : J[o * ldj + t];
      acc += m * src[base + t * stride];
    }
    out[idx] = accumulate ? out[idx] + acc : acc;
  }
}

template <typename T>
__global__ void k_contract_axis(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ J, int64_t Ne,
                                int d0, int d1, int d2, int axis, int nout, int ldj, int transpose, int accumulate) {
  pdl_entry();
  contract_axis_body<T>(plain_block(), in, out, J, Ne, d0, d1, d2, axis, nout, ldj, transpose, accumulate);
}

template <typename T>
cudaError_t contract(const mg_ctx* c, const T* in, T* out, const T* J, int d0, int d1, int d2, int axis, int nout,
                     int ldj, int transpose, int accumulate) {
  int o0 = d0, o1 = d1, o2 = d2;
  if (axis == 0) o0 = nout; else if (axis == 1) o1 = nout; else o2 = nout;
  int64_t total = c->Ne * (int64_t)o0 * o1 * o2;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  launch_pdl<kTwinType<T> ? &contract_axis_body<T> : nullptr>(k_contract_axis<T>, (int)blocks, 256, 0, c->stream, in,
                                                              out, J, c->Ne, d0, d1, d2, axis, nout, ldj, transpose,
                                                              accumulate);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// Even/odd product y = A x for a centro-symmetric NO x NI matrix given as its
// even part AE ((NO+1)/2 x (NI+1)/2) and odd part AO (NO/2 x NI/2):
//   e_t = x_t + x_{NI-1-t}, o_t = x_t - x_{NI-1-t} (t < NI/2), e_{NI/2} = x_{NI/2} (NI odd),
//   y_a = E_a + O_a, y_{NO-1-a} = E_a - O_a, y_{NO/2} = E_{NO/2} (NO odd).
// The interpolation matrix J (order P_l nodes x order P_{l-1} basis) is
// centro-symmetric because both GLL point sets are symmetric about 0.
template <typename T, int NO, int NI>
__device__ __forceinline__ void cs_matvec(const T* __restrict__ AE, const T* __restrict__ AO, const T (&x)[NI],
                                          T (&y)[NO]) {
  constexpr int hi = NI / 2, ho = NO / 2, nei = (NI + 1) / 2, neo = (NO + 1) / 2;
  T e[nei], o[hi > 0 ? hi : 1];
#pragma unroll
  for (int t = 0; t < hi; ++t) {
    e[t] = x[t] + x[NI - 1 - t];
    o[t] = x[t] - x[NI - 1 - t];
  }
  if (NI & 1) e[nei - 1] = x[hi];
#pragma unroll
  for (int a = 0; a < neo; ++a) {
    T E = AE[a * nei] * e[0];
#pragma unroll
    for (int t = 1; t < nei; ++t) E += AE[a * nei + t] * e[t];
    if (a < ho) {
      T O = AO[a * hi] * o[0];
#pragma unroll
      for (int t = 1; t < hi; ++t) O += AO[a * hi + t] * o[t];
      y[a] = E + O;
      y[NO - 1 - a] = E - O;
    } else {
      y[a] = E;
    }
  }
}

// Even / odd parts of the centro-symmetric matrix A (NO x NI, A[o][t] = get(o, t)).
template <typename T, int NO, int NI, typename Get>
__device__ void cs_split(Get get, T* AE, T* AO) {
  constexpr int hi = NI / 2, nei = (NI + 1) / 2, neo = (NO + 1) / 2, ho = NO / 2;
  for (int idx = threadIdx.x; idx < neo * nei; idx += blockDim.x) {
    const int a = idx / nei, t = idx % nei;
    AE[idx] = (t < hi) ? (T)0.5 * (get(a, t) + get(a, NI - 1 - t)) : get(a, t);
  }
  for (int idx = threadIdx.x; idx < ho * hi; idx += blockDim.x) {
    const int a = idx / hi, t = idx % hi;
    AO[idx] = (T)0.5 * (get(a, t) - get(a, NI - 1 - t));
  }
}

// Fused prolongation u_f += (J (x) J (x) J) u_c, TE elements per block pass
// (enough for the z pass to occupy the block's 256 threads), intermediates in
// shared memory.
template <int NF>
struct TrShape {
  static constexpr int te = 256 / (NF * NF) > 0 ? 256 / (NF * NF) : 1;  // elements per block pass
};

template <typename T, int NF, int NC>
__device__ __forceinline__ void prolong_fused_body(BlockIdx bi_, const T* __restrict__ uc, T* __restrict__ uf,
                                                   const T* __restrict__ J, int64_t Ne) {
  constexpr int nei = (NC + 1) / 2, neo = (NF + 1) / 2, TE = TrShape<NF>::te;
  constexpr int nB = NF * NC * NC, nC = NF * NF * NC;
  __shared__ T sE[neo * nei], sO[(NF / 2) * (NC / 2) + 1];
  __shared__ T sB[TE * nB], sC[TE * nC];
  cs_split<T, NF, NC>([&](int o, int t) { return J[o * NC + t]; }, sE, sO);
  __syncthreads();
  for (int64_t e0 = (int64_t)bi_.b * TE; e0 < Ne; e0 += (int64_t)bi_.g * TE) {
    const int cnt = (int)(Ne - e0 < TE ? Ne - e0 : TE);
    for (int w = threadIdx.x; w < cnt * NC * NC; w += blockDim.x) {  // x: (j,k) lines
      const int g = w / (NC * NC), ln = w - g * (NC * NC);
      const T* x0 = uc + (e0 + g) * (NC * NC * NC);
      T x[NC], y[NF];
#pragma unroll
      for (int t = 0; t < NC; ++t) x[t] = x0[t + NC * ln];
      cs_matvec<T, NF, NC>(sE, sO, x, y);
#pragma unroll
      for (int a = 0; a < NF; ++a) sB[g * nB + a + NF * ln] = y[a];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < cnt * NF * NC; w += blockDim.x) {  // y: (a,k) lines
      const int g = w / (NF * NC), ln = w - g * (NF * NC);
      const int a = ln % NF, k = ln / NF;
      T x[NC], y[NF];
#pragma unroll
      for (int t = 0; t < NC; ++t) x[t] = sB[g * nB + a + NF * (t + NC * k)];
      cs_matvec<T, NF, NC>(sE, sO, x, y);
#pragma unroll
      for (int b = 0; b < NF; ++b) sC[g * nC + a + NF * (b + NF * k)] = y[b];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < cnt * NF * NF; w += blockDim.x) {  // z: (a,b) lines, accumulate
      const int g = w / (NF * NF), ln = w - g * (NF * NF);
      T* out = uf + (e0 + g) * (NF * NF * NF);
      T x[NC], y[NF];
#pragma unroll
      for (int t = 0; t < NC; ++t) x[t] = sC[g * nC + ln + NF * NF * t];
      cs_matvec<T, NF, NC>(sE, sO, x, y);
#pragma unroll
      for (int c = 0; c < NF; ++c) out[ln + NF * NF * c] += y[c];
    }
    __syncthreads();
  }
}

template <typename T, int NF, int NC>
__global__ void __launch_bounds__(256) k_prolong_fused(const T* __restrict__ uc, T* __restrict__ uf,
                                  const T* __restrict__ J, int64_t Ne) {
  pdl_entry();
  prolong_fused_body<T, NF, NC>(plain_block(), uc, uf, J, Ne);
}

// Fused restriction f_c = (J^T (x) J^T (x) J^T) r_f, TE elements per block pass.
template <typename T, int NF, int NC>
__device__ __forceinline__ void restrict_fused_body(BlockIdx bi_, const T* __restrict__ rf, T* __restrict__ fc,
                                                    const T* __restrict__ J, int64_t Ne) {
  constexpr int nei = (NF + 1) / 2, neo = (NC + 1) / 2, TE = TrShape<NF>::te;
  constexpr int nB = NF * NC * NC, nC = NF * NF * NC;
  __shared__ T sE[neo * nei], sO[(NC / 2) * (NF / 2) + 1];
  __shared__ T sB[TE * nB], sC[TE * nC];
  cs_split<T, NC, NF>([&](int o, int t) { return J[t * NC + o]; }, sE, sO);
  __syncthreads();
  for (int64_t e0 = (int64_t)bi_.b * TE; e0 < Ne; e0 += (int64_t)bi_.g * TE) {
    const int cnt = (int)(Ne - e0 < TE ? Ne - e0 : TE);
    for (int w = threadIdx.x; w < cnt * NF * NF; w += blockDim.x) {  // z: (a,b) lines
      const int g = w / (NF * NF), ln = w - g * (NF * NF);
      const T* x0 = rf + (e0 + g) * (NF * NF * NF);
      T x[NF], y[NC];
#pragma unroll
      for (int t = 0; t < NF; ++t) x[t] = x0[ln + NF * NF * t];
      cs_matvec<T, NC, NF>(sE, sO, x, y);
#pragma unroll
      for (int k = 0; k < NC; ++k) sC[g * nC + ln + NF * NF * k] = y[k];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < cnt * NF * NC; w += blockDim.x) {  // y: (a,k) lines
      const int g = w / (NF * NC), ln = w - g * (NF * NC);
      const int a = ln % NF, k = ln / NF;
      T x[NF], y[NC];
#pragma unroll
      for (int t = 0; t < NF; ++t) x[t] = sC[g * nC + a + NF * (t + NF * k)];
      cs_matvec<T, NC, NF>(sE, sO, x, y);
#pragma unroll
      for (int j = 0; j < NC; ++j) sB[g * nB + a + NF * (j + NC * k)] = y[j];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < cnt * NC * NC; w += blockDim.x) {  // x: (j,k) lines
      const int g = w / (NC * NC), ln = w - g * (NC * NC);
      T* out = fc + (e0 + g) * (NC * NC * NC);
      T x[NF], y[NC];
#pragma unroll
      for (int t = 0; t < NF; ++t) x[t] = sB[g * nB + t + NF * ln];
      cs_matvec<T, NC, NF>(sE, sO, x, y);
#pragma unroll
      for (int i = 0; i < NC; ++i) out[i + NC * ln] = y[i];
    }
    __syncthreads();
  }
}

template <typename T, int NF, int NC>
__global__ void __launch_bounds__(256) k_restrict_fused(const T* __restrict__ rf, T* __restrict__ fc,
                                  const T* __restrict__ J, int64_t Ne) {
  pdl_entry();
  restrict_fused_body<T, NF, NC>(plain_block(), rf, fc, J, Ne);
}

// One-axis contraction with the even / odd halves of the centro-symmetric 1D
// matrix in the kernel's parameter space (order 32 in FP32, where the fused
// kernel's element block does not fit shared memory and the generic kernel
// above reloads a matrix entry for every multiply-add): one thread per line
// along AXIS of every element, NI inputs in, NO outputs out (added to the
// output with ACC), the products of cs_matvec.
template <typename T, int NO, int NI>
struct TrCArgs {
  static constexpr int nei = (NI + 1) / 2, hi = NI / 2, neo = (NO + 1) / 2, ho = NO / 2;
  const T* in;
  T* out;
  int64_t Ne;
  int d0, d1, d2;  // input extents per element, x fastest
  T ae[neo * nei];
  T ao[(ho > 0 ? ho : 1) * (hi > 0 ? hi : 1)];
};

template <typename T, int NO, int NI, int AXIS, bool ACC>
__global__ void __launch_bounds__(256) k_contract_c(const __grid_constant__ TrCArgs<T, NO, NI> a) {
  pdl_entry();
  const int o0 = AXIS == 0 ? NO : a.d0, o1 = AXIS == 1 ? NO : a.d1, o2 = AXIS == 2 ? NO : a.d2;
  const int nl = AXIS == 0 ? a.d1 * a.d2 : (AXIS == 1 ? a.d0 * a.d2 : a.d0 * a.d1);
  const int64_t gl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t e = gl / nl;
  if (e >= a.Ne) return;
  const int l = (int)(gl - e * nl);
  int ib, is, ob, os;
  if (AXIS == 0) {
    const int b = l % a.d1, c = l / a.d1;
    ib = a.d0 * (b + a.d1 * c); is = 1; ob = o0 * (b + o1 * c); os = 1;
  } else if (AXIS == 1) {
    const int x = l % a.d0, c = l / a.d0;
    ib = x + a.d0 * a.d1 * c; is = a.d0; ob = x + o0 * o1 * c; os = o0;
  } else {
    const int x = l % a.d0, b = l / a.d0;
    ib = x + a.d0 * b; is = a.d0 * a.d1; ob = x + o0 * b; os = o0 * o1;
  }
  const T* src = a.in + e * ((int64_t)a.d0 * a.d1 * a.d2) + ib;
  T* dst = a.out + e * ((int64_t)o0 * o1 * o2) + ob;
  T x[NI], y[NO];
#pragma unroll
  for (int t = 0; t < NI; ++t) x[t] = src[t * is];
  cs_matvec<T, NO, NI>(a.ae, a.ao, x, y);
#pragma unroll
  for (int t = 0; t < NO; ++t) dst[t * os] = ACC ? dst[t * os] + y[t] : y[t];
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

template <int NF>
inline int fused_blocks(int64_t Ne) {
  const int64_t groups = (Ne + TrShape<NF>::te - 1) / TrShape<NF>::te;
  return (int)(groups < 152 * 8 ? groups : 152 * 8);
}

// Halves of A (NO x NI, A[o][t] = J[o NC + t] for the prolongation, J[t NC + o]
// for the restriction) from the level's FP32 table, as cs_split forms them.
template <int NO, int NI>
void fill_trc(const mg_ctx* c, int l, bool transpose, TrCArgs<float, NO, NI>& a) {
  using A = TrCArgs<float, NO, NI>;
  const int nc = c->lev[l - 1].n;
  const float* J = c->tab32_host.data() + c->lev[l].J;
  auto get = [&](int o, int t) { return transpose ? J[t * nc + o] : J[o * nc + t]; };
  for (int o = 0; o < A::neo; ++o)
    for (int t = 0; t < A::nei; ++t)
      a.ae[o * A::nei + t] = (t < A::hi) ? 0.5f * (get(o, t) + get(o, NI - 1 - t)) : get(o, t);
  for (int o = 0; o < A::ho; ++o)
    for (int t = 0; t < A::hi; ++t) a.ao[o * A::hi + t] = 0.5f * (get(o, t) - get(o, NI - 1 - t));
}

template <int NO, int NI, int AXIS, bool ACC>
cudaError_t contract_c(const mg_ctx* c, TrCArgs<float, NO, NI>& a, const float* in, float* out, int d0, int d1,
                       int d2) {
  a.in = in;
  a.out = out;
  a.Ne = c->Ne;
  a.d0 = d0;
  a.d1 = d1;
  a.d2 = d2;
  const int nl = AXIS == 0 ? d1 * d2 : (AXIS == 1 ? d0 * d2 : d0 * d1);
  const int64_t blocks = (c->Ne * nl + 255) / 256;
  launch_pdl(k_contract_c<float, NO, NI, AXIS, ACC>, (int)blocks, 256, 0, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}


template <typename T, int NF, int NC>
cudaError_t restrict_fused(const mg_ctx* c, const T* r_fine, T* f_coarse, const T* J) {
  launch_pdl<kTwinType<T> ? &restrict_fused_body<T, NF, NC> : nullptr, 256>(
      k_restrict_fused<T, NF, NC>, fused_blocks<NF>(c->Ne), 256, 0, c->stream, r_fine, f_coarse, J, c->Ne);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T, int NF, int NC>
cudaError_t prolong_fused(const mg_ctx* c, const T* u_coarse, T* u_fine, const T* J) {
  launch_pdl<kTwinType<T> ? &prolong_fused_body<T, NF, NC> : nullptr, 256>(
      k_prolong_fused<T, NF, NC>, fused_blocks<NF>(c->Ne), 256, 0, c->stream, u_coarse, u_fine, J, c->Ne);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const mg_ctx* c, int l, const T* r_fine, T* f_coarse) {
  const int nf = c->lev[l].n, nc = c->lev[l - 1].n;
  const T* J = table_of<T>(c) + c->lev[l].J;
  switch (nf) {
    case 3: return restrict_fused<T, 3, 2>(c, r_fine, f_coarse, J);
    case 5: return restrict_fused<T, 5, 3>(c, r_fine, f_coarse, J);
    case 9: return restrict_fused<T, 9, 5>(c, r_fine, f_coarse, J);
    case 17: return restrict_fused<T, 17, 9>(c, r_fine, f_coarse, J);
    default: break;
  }
  T* t1 = static_cast<T*>(c->ws.corr);
  T* t2 = t1 + c->Ne * (int64_t)nf * nf * nc;
  cudaError_t e;
  if constexpr (std::is_same<T, float>::value) {
    if (nf == 33 && nc == 17 && launch_recorder() == nullptr && !c->tab32_host.empty()) {
      TrCArgs<float, 17, 33> a;
      fill_trc<17, 33>(c, l, true, a);
      if ((e = contract_c<17, 33, 2, false>(c, a, r_fine, t1, nf, nf, nf)) != cudaSuccess) return e;
      if ((e = contract_c<17, 33, 1, false>(c, a, t1, t2, nf, nf, nc)) != cudaSuccess) return e;
      return contract_c<17, 33, 0, false>(c, a, t2, f_coarse, nf, nc, nc);
    }
  }
  // z: (nf, nf, nf) -> (nf, nf, nc); y: -> (nf, nc, nc); x: -> (nc, nc, nc)
  if ((e = contract<T>(c, r_fine, t1, J, nf, nf, nf, 2, nc, nc, 1, 0)) != cudaSuccess) return e;
  if ((e = contract<T>(c, t1, t2, J, nf, nf, nc, 1, nc, nc, 1, 0)) != cudaSuccess) return e;
  return contract<T>(c, t2, f_coarse, J, nf, nc, nc, 0, nc, nc, 1, 0);
}

template <typename T>
cudaError_t launch_prolong(const mg_ctx* c, int l, const T* u_coarse, T* u_fine) {
  const int nf = c->lev[l].n, nc = c->lev[l - 1].n;
  const T* J = table_of<T>(c) + c->lev[l].J;
  switch (nf) {
    case 3: return prolong_fused<T, 3, 2>(c, u_coarse, u_fine, J);
    case 5: return prolong_fused<T, 5, 3>(c, u_coarse, u_fine, J);
    case 9: return prolong_fused<T, 9, 5>(c, u_coarse, u_fine, J);
    case 17: return prolong_fused<T, 17, 9>(c, u_coarse, u_fine, J);
    default: break;
  }
  T* t1 = static_cast<T*>(c->ws.corr);
  T* t2 = t1 + c->Ne * (int64_t)nf * nc * nc;
  cudaError_t e;
  if constexpr (std::is_same<T, float>::value) {
    if (nf == 33 && nc == 17 && launch_recorder() == nullptr && !c->tab32_host.empty()) {
      TrCArgs<float, 33, 17> a;
      fill_trc<33, 17>(c, l, false, a);
      if ((e = contract_c<33, 17, 0, false>(c, a, u_coarse, t1, nc, nc, nc)) != cudaSuccess) return e;
      if ((e = contract_c<33, 17, 1, false>(c, a, t1, t2, nf, nc, nc)) != cudaSuccess) return e;
      return contract_c<33, 17, 2, true>(c, a, t2, u_fine, nf, nf, nc);
    }
  }
  // x: (nc, nc, nc) -> (nf, nc, nc); y: -> (nf, nf, nc); z: -> (nf, nf, nf), accumulated
  if ((e = contract<T>(c, u_coarse, t1, J, nc, nc, nc, 0, nf, nc, 0, 0)) != cudaSuccess) return e;
  if ((e = contract<T>(c, t1, t2, J, nf, nc, nc, 1, nf, nc, 0, 0)) != cudaSuccess) return e;
  return contract<T>(c, t2, u_fine, J, nf, nf, nc, 2, nf, nc, 0, 1);
}

template cudaError_t launch_restrict<double>(const mg_ctx*, int, const double*, double*);
template cudaError_t launch_restrict<float>(const mg_ctx*, int, const float*, float*);
template cudaError_t launch_prolong<double>(const mg_ctx*, int, const double*, double*);
template cudaError_t launch_prolong<float>(const mg_ctx*, int, const float*, float*);
template cudaError_t launch_restrict<df64>(const mg_ctx*, int, const df64*, df64*);
template cudaError_t launch_prolong<df64>(const mg_ctx*, int, const df64*, df64*);

}  // namespace mgdg
