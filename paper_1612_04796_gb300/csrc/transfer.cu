// Polynomial transfers between levels (Section 3.2, Algorithm 1):
//   prolongation  u_l += I_l u_{l-1},    I_l = J (x) J (x) J per element,
//   restriction   f_{l-1} = I_l^T r_l,
// with J (n_f x n_c) the values of the order-P_{l-1} GLL Lagrange basis at the
// order-P_l GLL nodes (embedded interpolation).  Both are applied as three
// one-axis contractions (sum factorisation), one output value per thread,
// through the smoother's correction buffer as scratch.
#include "mg_internal.h"

namespace mgdg {
namespace {

// out[e][...o...] (+)= sum_t Mat(o, t) in[e][...t...] along `axis` of a
// per-element tensor with extents (d0, d1, d2), x fastest.
// Mat(o, t) = transpose ? J[t * ldj + o] : J[o * ldj + t].
template <typename T>
__global__ void k_contract_axis(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ J, int64_t Ne,
                                int d0, int d1, int d2, int axis, int nout, int ldj, int transpose, int accumulate) {
  int o0 = d0, o1 = d1, o2 = d2;
  if (axis == 0) o0 = nout; else if (axis == 1) o1 = nout; else o2 = nout;
  const int64_t in_sz = (int64_t)d0 * d1 * d2, out_sz = (int64_t)o0 * o1 * o2;
  const int64_t total = Ne * out_sz;
  const int nin = axis == 0 ? d0 : (axis == 1 ? d1 : d2);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
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
cudaError_t contract(const mg_ctx* c, const T* in, T* out, const T* J, int d0, int d1, int d2, int axis, int nout,
                     int ldj, int transpose, int accumulate) {
  int o0 = d0, o1 = d1, o2 = d2;
  if (axis == 0) o0 = nout; else if (axis == 1) o1 = nout; else o2 = nout;
  int64_t total = c->Ne * (int64_t)o0 * o1 * o2;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_contract_axis<T><<<(int)blocks, 256, 0, c->stream>>>(in, out, J, c->Ne, d0, d1, d2, axis, nout, ldj, transpose,
                                                         accumulate);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T>
const T* table_of(const mg_ctx* c);
template <>
const double* table_of<double>(const mg_ctx* c) { return c->ws.tab64; }
template <>
const float* table_of<float>(const mg_ctx* c) { return c->ws.tab32; }

}  // namespace

template <typename T>
cudaError_t launch_restrict(const mg_ctx* c, int l, const T* r_fine, T* f_coarse) {
  const int nf = c->lev[l].n, nc = c->lev[l - 1].n;
  const T* J = table_of<T>(c) + c->lev[l].J;
  T* t1 = static_cast<T*>(c->ws.corr);
  T* t2 = t1 + c->Ne * (int64_t)nf * nf * nc;
  cudaError_t e;
  // z: (nf, nf, nf) -> (nf, nf, nc); y: -> (nf, nc, nc); x: -> (nc, nc, nc)
  if ((e = contract<T>(c, r_fine, t1, J, nf, nf, nf, 2, nc, nc, 1, 0)) != cudaSuccess) return e;
  if ((e = contract<T>(c, t1, t2, J, nf, nf, nc, 1, nc, nc, 1, 0)) != cudaSuccess) return e;
  return contract<T>(c, t2, f_coarse, J, nf, nc, nc, 0, nc, nc, 1, 0);
}

template <typename T>
cudaError_t launch_prolong(const mg_ctx* c, int l, const T* u_coarse, T* u_fine) {
  const int nf = c->lev[l].n, nc = c->lev[l - 1].n;
  const T* J = table_of<T>(c) + c->lev[l].J;
  T* t1 = static_cast<T*>(c->ws.corr);
  T* t2 = t1 + c->Ne * (int64_t)nf * nc * nc;
  cudaError_t e;
  // x: (nc, nc, nc) -> (nf, nc, nc); y: -> (nf, nf, nc); z: -> (nf, nf, nf), accumulated
  if ((e = contract<T>(c, u_coarse, t1, J, nc, nc, nc, 0, nf, nc, 0, 0)) != cudaSuccess) return e;
  if ((e = contract<T>(c, t1, t2, J, nf, nc, nc, 1, nf, nc, 0, 0)) != cudaSuccess) return e;
  return contract<T>(c, t2, u_fine, J, nf, nf, nc, 2, nf, nc, 0, 1);
}

template cudaError_t launch_restrict<double>(const mg_ctx*, int, const double*, double*);
template cudaError_t launch_restrict<float>(const mg_ctx*, int, const float*, float*);
template cudaError_t launch_prolong<double>(const mg_ctx*, int, const double*, double*);
template cudaError_t launch_prolong<float>(const mg_ctx*, int, const float*, float*);

}  // namespace mgdg
