// Sum-factorised SIPG operator (Section 2, Eq. A):
//   A = Mz(x)My(x)Lx + Mz(x)Ly(x)Mx + Lz(x)My(x)Mx
// applied element by element.  Row block e of the 1D matrix L is
//   L_ee u_e + L_e,e-1 u_e-1 + L_e,e+1 u_e+1,
// where L_ee = (2/h) D^T W D plus the self terms of both faces and the
// neighbour couplings are rank-2 face terms (standard SIPG reading of Eq. ip):
//   (L_e,e-1 u_e-1)_i = delta_i0 (-mu a + g/2 b) - g/2 D0_i a,
//        a = u_e-1 at its node P, b = (D u_e-1) at its node P,
//   (L_e,e+1 u_e+1)_i = delta_iP (-mu c - g/2 d) + g/2 DP_i c,
//        c = u_e+1 at its node 0, d = (D u_e+1) at its node 0,
// with g = 2/h, D0 / DP the first / last row of the reference
// differentiation matrix.  One thread per output DOF; the element and its
// face neighbours are read through L1/L2.
#include "mg_internal.h"

namespace mgdg {
namespace {

template <typename T>
struct OpArgs {
  const T* tab;
  const T* u;
  const T* f;
  T* out;
  int64_t Ne;
  int nx, ny, nz, n, residual;
  int64_t lee[3], mass[3], d0, dp;
  T g[3], mu[3];
};

template <typename T>
__global__ void __launch_bounds__(256) k_sipg(OpArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int n = a.n, n2 = n * n, n3 = n2 * n, P = n - 1;
  T* sL = sm;             // 3 n^2
  T* sM = sL + 3 * n2;    // 3 n
  T* sD0 = sM + 3 * n;    // n
  T* sDP = sD0 + n;       // n
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    sL[i] = a.tab[a.lee[0] + i];
    sL[n2 + i] = a.tab[a.lee[1] + i];
    sL[2 * n2 + i] = a.tab[a.lee[2] + i];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sM[i] = a.tab[a.mass[0] + i];
    sM[n + i] = a.tab[a.mass[1] + i];
    sM[2 * n + i] = a.tab[a.mass[2] + i];
    sD0[i] = a.tab[a.d0 + i];
    sDP[i] = a.tab[a.dp + i];
  }
  __syncthreads();
  const int64_t total = a.Ne * n3;
  const T half = (T)0.5;
  for (int64_t dof = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; dof < total;
       dof += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = dof / n3;
    const int loc = (int)(dof - e * n3);
    const int i = loc % n, j = (loc / n) % n, k = loc / n2;
    const int ex = (int)(e % a.nx), ey = (int)((e / a.nx) % a.ny), ez = (int)(e / ((int64_t)a.nx * a.ny));
    const T* ue = a.u + e * n3;
    T sx = 0, sy = 0, sz = 0;
    for (int t = 0; t < n; ++t) {
      sx += sL[i * n + t] * ue[t + n * (j + n * k)];
      sy += sL[n2 + j * n + t] * ue[i + n * (t + n * k)];
      sz += sL[2 * n2 + k * n + t] * ue[i + n * (j + n * t)];
    }
    // x faces
    {
      const int64_t eL = (ex == 0 ? ex + a.nx - 1 : ex - 1) + a.nx * (ey + (int64_t)a.ny * ez);
      const int64_t eR = (ex == a.nx - 1 ? 0 : ex + 1) + a.nx * (ey + (int64_t)a.ny * ez);
      const T* uL = a.u + eL * n3 + n * (j + n * k);
      const T* uR = a.u + eR * n3 + n * (j + n * k);
      const T av = uL[P], cv = uR[0];
      const T g = a.g[0], mu = a.mu[0];
      sx += g * half * (sDP[i] * cv - sD0[i] * av);
      if (i == 0) {
        T b = 0;
        for (int t = 0; t < n; ++t) b += sDP[t] * uL[t];
        sx += g * half * b - mu * av;
      }
      if (i == P) {
        T d = 0;
        for (int t = 0; t < n; ++t) d += sD0[t] * uR[t];
        sx -= mu * cv + g * half * d;
      }
    }
    // y faces
    {
      const int64_t eL = ex + a.nx * ((ey == 0 ? ey + a.ny - 1 : ey - 1) + (int64_t)a.ny * ez);
      const int64_t eR = ex + a.nx * ((ey == a.ny - 1 ? 0 : ey + 1) + (int64_t)a.ny * ez);
      const T* uL = a.u + eL * n3 + i + n2 * k;
      const T* uR = a.u + eR * n3 + i + n2 * k;
      const T av = uL[n * P], cv = uR[0];
      const T g = a.g[1], mu = a.mu[1];
      sy += g * half * (sDP[j] * cv - sD0[j] * av);
      if (j == 0) {
        T b = 0;
        for (int t = 0; t < n; ++t) b += sDP[t] * uL[n * t];
        sy += g * half * b - mu * av;
      }
      if (j == P) {
        T d = 0;
        for (int t = 0; t < n; ++t) d += sD0[t] * uR[n * t];
        sy -= mu * cv + g * half * d;
      }
    }
    // z faces
    {
      const int64_t eL = ex + a.nx * (ey + (int64_t)a.ny * (ez == 0 ? ez + a.nz - 1 : ez - 1));
      const int64_t eR = ex + a.nx * (ey + (int64_t)a.ny * (ez == a.nz - 1 ? 0 : ez + 1));
      const T* uL = a.u + eL * n3 + i + n * j;
      const T* uR = a.u + eR * n3 + i + n * j;
      const T av = uL[n2 * P], cv = uR[0];
      const T g = a.g[2], mu = a.mu[2];
      sz += g * half * (sDP[k] * cv - sD0[k] * av);
      if (k == 0) {
        T b = 0;
        for (int t = 0; t < n; ++t) b += sDP[t] * uL[n2 * t];
        sz += g * half * b - mu * av;
      }
      if (k == P) {
        T d = 0;
        for (int t = 0; t < n; ++t) d += sD0[t] * uR[n2 * t];
        sz -= mu * cv + g * half * d;
      }
    }
    const T mx = sM[i], my = sM[n + j], mz = sM[2 * n + k];
    const T Au = mz * (my * sx + mx * sy) + my * mx * sz;
    a.out[dof] = a.residual ? a.f[dof] - Au : Au;
  }
}

template <typename T>
const T* table_of(const mg_ctx* c);
template <>
const double* table_of<double>(const mg_ctx* c) { return c->ws.tab64; }
template <>
const float* table_of<float>(const mg_ctx* c) { return c->ws.tab32; }

}  // namespace

template <typename T>
cudaError_t launch_sipg(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual) {
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
    a.lee[d] = lv.t[d].lee;
    a.mass[d] = lv.t[d].mass;
    a.g[d] = (T)lv.g[d];
    a.mu[d] = (T)lv.mu[d];
  }
  a.d0 = lv.t[0].d0;
  a.dp = lv.t[0].dp;
  const int n = lv.n;
  size_t smem = sizeof(T) * (3 * n * n + 5 * n);
  int64_t total = c->Ne * (int64_t)n * n * n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_sipg<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_sipg<T><<<(int)blocks, 256, smem, c->stream>>>(a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template cudaError_t launch_sipg<double>(const mg_ctx*, int, const double*, const double*, double*, int);
template cudaError_t launch_sipg<float>(const mg_ctx*, int, const float*, const float*, float*, int);

}  // namespace mgdg
