// Weighted overlapping additive Schwarz smoother (Section 3.1).
//
// k_fdm: one thread block per element-centred subdomain s.  The subdomain
// residual r_s = R_s r (m^3 values from the element and its 26 neighbours:
// N_O node layers per side) is gathered into the subdomain's slot of the
// correction buffer; the fast diagonalisation
//   du_s = (Sz(x)Sy(x)Sx) (I(x)I(x)Lx + I(x)Ly(x)I + Lz(x)I(x)I)^{-1} (Sz^T(x)Sy^T(x)Sx^T) r_s
// is applied in place, one 1D line per thread per direction, with the weights
// W_s = Wz(x)Wy(x)Wx folded into the backward factors (rows of S scaled by w).
//
// k_scatter: u += sum_s R_s^T (W_s du_s) (Eq. correction:global) evaluated per
// output DOF: every DOF sums the <= 8 (<= 27 at the widest overlap) subdomain
// values that cover it in a fixed order, so the result is deterministic and
// no atomics are needed.
#include "mg_internal.h"

namespace mgdg {
namespace {

template <typename T>
struct FdmArgs {
  const T* tab;
  const T* r;
  T* corr;
  int64_t Ne;
  int nx, ny, nz, n, m, no;
  int64_t S[3], SW[3], dinv;
};

// Subdomain line position a -> (element offset, node index).
__device__ __forceinline__ void sub_node(int a, int n, int no, int* de, int* ii) {
  if (a < no) { *de = -1; *ii = n - no + a; }
  else if (a < no + n) { *de = 0; *ii = a - no; }
  else { *de = 1; *ii = a - no - n; }
}

__device__ __forceinline__ int wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// In-place 1D contraction of all m^2 lines of the tile along `axis`:
// forward  (backward == 0): v[p] = sum_a S[a][p] x[a]      (S^T)
// backward (backward == 1): v[a] = sum_p SW[a][p] x[p]     (diag(w) S)
template <typename T>
__device__ void contract_lines(T* tile, const T* mat, int m, int axis, int backward) {
  const int m2 = m * m;
  const int stride = axis == 0 ? 1 : (axis == 1 ? m : m2);
  T line[kMaxM];
  for (int ln = threadIdx.x; ln < m2; ln += blockDim.x) {
    const int u = ln % m, v = ln / m;
    int base;
    if (axis == 0) base = m * (u + m * v);
    else if (axis == 1) base = u + m2 * v;
    else base = u + m * v;
    for (int a = 0; a < m; ++a) line[a] = tile[base + a * stride];
    for (int p = 0; p < m; ++p) {
      T acc = 0;
      if (!backward) {
        for (int a = 0; a < m; ++a) acc += mat[a * m + p] * line[a];
      } else {
        for (int q = 0; q < m; ++q) acc += mat[p * m + q] * line[q];
      }
      tile[base + p * stride] = acc;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fdm(FdmArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int m = a.m, m2 = m * m, m3 = m2 * m, n = a.n, n3 = n * n * n, no = a.no;
  T* sS = sm;              // 3 m^2
  T* sSW = sS + 3 * m2;    // 3 m^2
  for (int i = threadIdx.x; i < m2; i += blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      sS[d * m2 + i] = a.tab[a.S[d] + i];
      sSW[d * m2 + i] = a.tab[a.SW[d] + i];
    }
  }
  __syncthreads();
  for (int64_t s = blockIdx.x; s < a.Ne; s += gridDim.x) {
    const int sx = (int)(s % a.nx), sy = (int)((s / a.nx) % a.ny), sz = (int)(s / ((int64_t)a.nx * a.ny));
    T* tile = a.corr + s * (int64_t)m3;
    // gather r_s = R_s r
    for (int idx = threadIdx.x; idx < m3; idx += blockDim.x) {
      const int ia = idx % m, ib = (idx / m) % m, ic = idx / m2;
      int dx, ix, dy, iy, dz, iz;
      sub_node(ia, n, no, &dx, &ix);
      sub_node(ib, n, no, &dy, &iy);
      sub_node(ic, n, no, &dz, &iz);
      const int64_t e = wrap(sx + dx, a.nx) + a.nx * (wrap(sy + dy, a.ny) + (int64_t)a.ny * wrap(sz + dz, a.nz));
      tile[idx] = a.r[e * n3 + ix + n * (iy + n * iz)];
    }
    __syncthreads();
    contract_lines(tile, sS, m, 0, 0);
    __syncthreads();
    contract_lines(tile, sS + m2, m, 1, 0);
    __syncthreads();
    contract_lines(tile, sS + 2 * m2, m, 2, 0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < m3; idx += blockDim.x) tile[idx] *= a.tab[a.dinv + idx];
    __syncthreads();
    contract_lines(tile, sSW + 2 * m2, m, 2, 1);
    __syncthreads();
    contract_lines(tile, sSW + m2, m, 1, 1);
    __syncthreads();
    contract_lines(tile, sSW, m, 0, 1);
    __syncthreads();
  }
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ corr, T* __restrict__ u, int64_t Ne, int nx, int ny, int nz, int n,
                          int m, int no, int accumulate) {
  const int n3 = n * n * n, m2 = m * m, m3 = m2 * m;
  const int64_t total = Ne * n3;
  for (int64_t dof = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; dof < total;
       dof += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = dof / n3;
    const int loc = (int)(dof - e * n3);
    const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    // per direction: covering subdomains (offset, position), fixed order -1, 0, +1
    int ox[3], px[3], cx = 0, oy[3], py[3], cy = 0, oz[3], pz[3], cz = 0;
    if (i < no) { ox[cx] = -1; px[cx++] = no + n + i; }
    ox[cx] = 0; px[cx++] = no + i;
    if (i >= n - no) { ox[cx] = 1; px[cx++] = i - (n - no); }
    if (j < no) { oy[cy] = -1; py[cy++] = no + n + j; }
    oy[cy] = 0; py[cy++] = no + j;
    if (j >= n - no) { oy[cy] = 1; py[cy++] = j - (n - no); }
    if (k < no) { oz[cz] = -1; pz[cz++] = no + n + k; }
    oz[cz] = 0; pz[cz++] = no + k;
    if (k >= n - no) { oz[cz] = 1; pz[cz++] = k - (n - no); }
    T sum = 0;
    for (int c = 0; c < cz; ++c) {
      const int64_t zz = wrap(ez + oz[c], nz);
      for (int b = 0; b < cy; ++b) {
        const int64_t yy = wrap(ey + oy[b], ny);
        for (int q = 0; q < cx; ++q) {
          const int64_t s = wrap(ex + ox[q], nx) + nx * (yy + ny * zz);
          sum += corr[s * m3 + px[q] + m * (py[b] + m * pz[c])];
        }
      }
    }
    u[dof] = accumulate ? u[dof] + sum : sum;
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
cudaError_t launch_fdm(const mg_ctx* c, int l, const T* r) {
  const LevelInfo& lv = c->lev[l];
  FdmArgs<T> a;
  a.tab = table_of<T>(c);
  a.r = r;
  a.corr = static_cast<T*>(c->ws.corr);
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.n = lv.n;
  a.m = lv.m;
  a.no = lv.no;
  for (int d = 0; d < 3; ++d) {
    a.S[d] = lv.t[d].S;
    a.SW[d] = lv.t[d].SW;
  }
  a.dinv = lv.dinv;
  size_t smem = sizeof(T) * 6 * lv.m * lv.m;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fdm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int threads = lv.m * lv.m >= 256 ? 256 : 128;
  int64_t blocks = c->Ne < 152 * 8 ? c->Ne : 152 * 8;
  k_fdm<T><<<(int)blocks, threads, smem, c->stream>>>(a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter(const mg_ctx* c, int l, T* u, int accumulate) {
  const LevelInfo& lv = c->lev[l];
  int64_t total = lv.N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scatter<T><<<(int)blocks, 256, 0, c->stream>>>(static_cast<const T*>(c->ws.corr), u, c->Ne, c->ne[0], c->ne[1],
                                                    c->ne[2], lv.n, lv.m, lv.no, accumulate);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template cudaError_t launch_fdm<double>(const mg_ctx*, int, const double*);
template cudaError_t launch_fdm<float>(const mg_ctx*, int, const float*);
template cudaError_t launch_scatter<double>(const mg_ctx*, int, double*, int);
template cudaError_t launch_scatter<float>(const mg_ctx*, int, float*, int);

}  // namespace mgdg
