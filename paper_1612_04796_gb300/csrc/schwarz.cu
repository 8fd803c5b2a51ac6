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
#include <algorithm>
#include <type_traits>

#include "fdm_tmpl.cuh"

namespace mgdg {

MGDG_FDM_EXTERN(3) MGDG_FDM_EXTERN(5) MGDG_FDM_EXTERN(7) MGDG_FDM_EXTERN(9) MGDG_FDM_EXTERN(11)
MGDG_FDM_EXTERN(13) MGDG_FDM_EXTERN(15) MGDG_FDM_EXTERN(17) MGDG_FDM_EXTERN(19) MGDG_FDM_EXTERN(21)
MGDG_FDM_EXTERN(23) MGDG_FDM_EXTERN(25) MGDG_FDM_EXTERN(27) MGDG_FDM_EXTERN(29) MGDG_FDM_EXTERN(31)
MGDG_FDM_EXTERN(33) MGDG_FDM_EXTERN(35)
MGDG_FDM_DF_WIDTHS(MGDG_FDM_EXTERN_DF)

namespace {

using mgdg::FdmArgs;

__device__ __forceinline__ void sub_node(int a, int n, int no, int* de, int* ii) { fdm_sub_node(a, n, no, de, ii); }
__device__ __forceinline__ int wrap(int x, int n) { return fdm_wrap(x, n); }

// Even/odd 1D transforms of one subdomain line (m = 2h+1, odd).  The
// eigenvectors of the reflection-symmetric line problem are even (columns
// p < h+1 of S) or odd (columns h+1 .. 2h), so with e_a = x_a + x_{m-1-a},
// o_a = x_a - x_{m-1-a} (a < h) and e_h = x_h:
//   forward  v_p     = sum_{a<=h} S[a][p] e_a          (p <= h)
//            v_{h+1+q} = sum_{a<h} S[a][h+1+q] o_a     (q < h)
//   backward x_a, x_{m-1-a} = E_a +- O_a, E_a = sum_{p<=h} SW[a][p] v_p,
//            O_a = sum_{q<h} SW[a][h+1+q] v_{h+1+q},  x_h = E_h.
// (h+1)^2 + h^2 multiply-adds and 2h additions instead of m^2.
template <typename T>
__device__ __forceinline__ void fwd_eo(T* x, const T* __restrict__ S, int m, T* __restrict__ out, int ost) {
  const int h = m >> 1, ne = h + 1;
  for (int a = 0; a < h; ++a) {
    const T xa = x[a], xb = x[m - 1 - a];
    x[a] = xa + xb;          // e_a
    x[m - 1 - a] = xa - xb;  // o_a stored at m-1-a
  }
  for (int p = 0; p < ne; ++p) {
    T acc = 0;
    for (int a = 0; a <= h; ++a) acc += S[a * m + p] * x[a];
    out[p * ost] = acc;
  }
  for (int q = 0; q < h; ++q) {
    T acc = 0;
    for (int a = 0; a < h; ++a) acc += S[a * m + ne + q] * x[m - 1 - a];
    out[(ne + q) * ost] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void bwd_eo(const T* v, const T* __restrict__ SW, int m, T* __restrict__ out, int ost) {
  const int h = m >> 1, ne = h + 1;
  for (int a = 0; a <= h; ++a) {
    T E = 0;
    for (int p = 0; p < ne; ++p) E += SW[a * m + p] * v[p];
    if (a < h) {
      T O = 0;
      for (int q = 0; q < h; ++q) O += SW[a * m + ne + q] * v[ne + q];
      out[a * ost] = E + O;
      out[(m - 1 - a) * ost] = E - O;
    } else {
      out[a * ost] = E;
    }
  }
}

// Run-time widths m_x, m_y, m_z (subdomains need not be cubic: with the "max"
// overlap of Table 2 every direction has its own N_O).  The tile of subdomain s
// is stored at corr + s m_x m_y m_z, node (a, b, c) at a + m_x (b + m_y c).
// The six 1D factors are staged in shared memory when they fit, else read
// through the cache from the table array.
template <typename T>
__device__ __forceinline__ void fdm_body(BlockIdx bi_, FdmArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int mx = a.md[0], my = a.md[1], mz = a.md[2], mxy = mx * my, mxyz = mxy * mz;
  const int n = a.n, n3 = n * n * n, nox = a.nod[0], noy = a.nod[1], noz = a.nod[2];
  const T* S[3];
  const T* SW[3];
  if (a.s_in_smem) {
    T* p = sm;
    for (int d = 0; d < 3; ++d) {
      const int md2 = a.md[d] * a.md[d];
      for (int i = threadIdx.x; i < md2; i += blockDim.x) {
        p[i] = a.tab[a.S[d] + i];
        p[md2 + i] = a.tab[a.SW[d] + i];
      }
      S[d] = p;
      SW[d] = p + md2;
      p += 2 * md2;
    }
    __syncthreads();
  } else {
    for (int d = 0; d < 3; ++d) {
      S[d] = a.tab + a.S[d];
      SW[d] = a.tab + a.SW[d];
    }
  }
  const T* __restrict__ dinv = a.tab + a.dinv;
  T x[kMaxM], v[kMaxM];
  for (int64_t s = bi_.b; s < a.Ne; s += bi_.g) {
    const int s32 = (int)s, sxy = s32 / a.nx;
    const int sx = s32 - sxy * a.nx, sy = sxy % a.ny, sz = sxy / a.ny;
    T* tile = a.corr + s * (int64_t)mxyz;
    const int64_t exl = wrap(sx - 1, a.nx), exr = wrap(sx + 1, a.nx);
    // pass 1: gather the x-lines of r_s = R_s r and transform them (forward, x)
    for (int ln = threadIdx.x; ln < my * mz; ln += blockDim.x) {
      const int b = ln % my, c = ln / my;
      int dy, iy, dz, iz;
      sub_node(b, n, noy, &dy, &iy);
      sub_node(c, n, noz, &dz, &iz);
      const int64_t row = a.nx * (wrap(sy + dy, a.ny) + (int64_t)a.ny * wrap(sz + dz, a.nz));
      const int loc = n * (iy + n * iz);
      const T* rl = a.r + (exl + row) * n3 + loc;
      const T* rc = a.r + (sx + row) * n3 + loc;
      const T* rr = a.r + (exr + row) * n3 + loc;
      for (int t = 0; t < nox; ++t) x[t] = rl[n - nox + t];
      for (int t = 0; t < n; ++t) x[nox + t] = rc[t];
      for (int t = 0; t < nox; ++t) x[nox + n + t] = rr[t];
      fwd_eo(x, S[0], mx, tile + mx * ln, 1);
    }
    __syncthreads();
    // pass 2: forward, y
    for (int ln = threadIdx.x; ln < mx * mz; ln += blockDim.x) {
      const int ia = ln % mx, c = ln / mx;
      T* line = tile + ia + mxy * c;
      for (int t = 0; t < my; ++t) x[t] = line[t * mx];
      fwd_eo(x, S[1], my, line, mx);
    }
    __syncthreads();
    // pass 3: forward z, divide by lam_x + lam_y + lam_z, backward z
    for (int ln = threadIdx.x; ln < mxy; ln += blockDim.x) {
      T* line = tile + ln;
      for (int t = 0; t < mz; ++t) x[t] = line[t * mxy];
      fwd_eo(x, S[2], mz, v, 1);
      for (int t = 0; t < mz; ++t) v[t] *= dinv[ln + t * mxy];
      bwd_eo(v, SW[2], mz, line, mxy);
    }
    __syncthreads();
    // pass 4: backward, y
    for (int ln = threadIdx.x; ln < mx * mz; ln += blockDim.x) {
      const int ia = ln % mx, c = ln / mx;
      T* line = tile + ia + mxy * c;
      for (int t = 0; t < my; ++t) v[t] = line[t * mx];
      bwd_eo(v, SW[1], my, line, mx);
    }
    __syncthreads();
    // pass 5: backward, x (weights folded into SW)
    for (int ln = threadIdx.x; ln < my * mz; ln += blockDim.x) {
      T* line = tile + mx * ln;
      for (int t = 0; t < mx; ++t) v[t] = line[t];
      bwd_eo(v, SW[0], mx, line, 1);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fdm(FdmArgs<T> a) {
  pdl_entry();
  fdm_body<T>(plain_block(), a);
}

// Subdomain geometry of the scatter: widths and layers per direction.
struct SubShape {
  int mx, my, mz, nox, noy, noz;
};

template <typename T>
__device__ __forceinline__ void scatter_body(BlockIdx bi_, const T* __restrict__ corr, T* __restrict__ u, int64_t Ne,
                                             int nx, int ny, int nz, int n, SubShape g, int accumulate) {
  const int n3 = n * n * n;
  const int64_t mxyz = (int64_t)g.mx * g.my * g.mz;
  const int64_t total = Ne * n3;
  for (int64_t dof = bi_.b * (int64_t)blockDim.x + threadIdx.x; dof < total;
       dof += (int64_t)bi_.g * blockDim.x) {
    const int e = (int)(dof / n3);
    const int loc = (int)(dof - (int64_t)e * n3);
    const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const int exy = e / nx;
    const int ex = e - exy * nx, ey = exy % ny, ez = exy / ny;
    // per direction: covering subdomains (offset, position), fixed order -1, 0, +1
    int ox[3], px[3], cx = 0, oy[3], py[3], cy = 0, oz[3], pz[3], cz = 0;
    if (i < g.nox) { ox[cx] = -1; px[cx++] = g.nox + n + i; }
    ox[cx] = 0; px[cx++] = g.nox + i;
    if (i >= n - g.nox) { ox[cx] = 1; px[cx++] = i - (n - g.nox); }
    if (j < g.noy) { oy[cy] = -1; py[cy++] = g.noy + n + j; }
    oy[cy] = 0; py[cy++] = g.noy + j;
    if (j >= n - g.noy) { oy[cy] = 1; py[cy++] = j - (n - g.noy); }
    if (k < g.noz) { oz[cz] = -1; pz[cz++] = g.noz + n + k; }
    oz[cz] = 0; pz[cz++] = g.noz + k;
    if (k >= n - g.noz) { oz[cz] = 1; pz[cz++] = k - (n - g.noz); }
    T sum = 0;
    for (int c = 0; c < cz; ++c) {
      const int64_t zz = wrap(ez + oz[c], nz);
      for (int b = 0; b < cy; ++b) {
        const int64_t yy = wrap(ey + oy[b], ny);
        for (int q = 0; q < cx; ++q) {
          const int64_t s = wrap(ex + ox[q], nx) + nx * (yy + ny * zz);
          sum += corr[s * mxyz + px[q] + g.mx * (py[b] + g.my * pz[c])];
        }
      }
    }
    u[dof] = accumulate ? u[dof] + sum : sum;
  }
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ corr, T* __restrict__ u, int64_t Ne, int nx, int ny, int nz, int n,
                          SubShape g, int accumulate) {
  pdl_entry();
  scatter_body<T>(plain_block(), corr, u, Ne, nx, ny, nz, n, g, accumulate);
}

// Same sum as k_scatter with compile-time n: one thread per DOF, the 27
// possible covering subdomains visited in the same fixed order (-1, 0, +1 per
// direction, x fastest) with predicates instead of per-DOF lists.
template <typename T, int N>
__device__ __forceinline__ void scatter_n_body(BlockIdx bi_, const T* __restrict__ corr, T* __restrict__ u, int64_t Ne,
                                               int nx, int ny, int nz, SubShape g, int accumulate) {
  constexpr int N3 = N * N * N;
  const int64_t mxyz = (int64_t)g.mx * g.my * g.mz;
  const int64_t total = Ne * N3;
  for (int64_t dof = bi_.b * (int64_t)blockDim.x + threadIdx.x; dof < total;
       dof += (int64_t)bi_.g * blockDim.x) {
    const int e = (int)(dof / N3);  // element indices fit in 32 bits
    const int loc = (int)(dof - (int64_t)e * N3);
    const int i = loc % N, j = (loc / N) % N, k = loc / (N * N);
    const int exy = e / nx;
    const int ex = e - exy * nx, ey = exy % ny, ez = exy / ny;
    // per direction and offset o (0: subdomain to the left, 1: own, 2: to the right):
    // covered?  position in that subdomain's line
    const bool vx0 = i < g.nox, vx2 = i >= N - g.nox, vy0 = j < g.noy, vy2 = j >= N - g.noy, vz0 = k < g.noz,
               vz2 = k >= N - g.noz;
    const int px[3] = {g.nox + N + i, g.nox + i, i - (N - g.nox)};
    const int py[3] = {g.noy + N + j, g.noy + j, j - (N - g.noy)};
    const int pz[3] = {g.noz + N + k, g.noz + k, k - (N - g.noz)};
    const int sxs[3] = {ex == 0 ? nx - 1 : ex - 1, ex, ex == nx - 1 ? 0 : ex + 1};
    const int sys[3] = {ey == 0 ? ny - 1 : ey - 1, ey, ey == ny - 1 ? 0 : ey + 1};
    const int szs[3] = {ez == 0 ? nz - 1 : ez - 1, ez, ez == nz - 1 ? 0 : ez + 1};
    T sum = 0;
#pragma unroll
    for (int oz = 0; oz < 3; ++oz) {
      if ((oz == 0 && !vz0) || (oz == 2 && !vz2)) continue;
#pragma unroll
      for (int oy = 0; oy < 3; ++oy) {
        if ((oy == 0 && !vy0) || (oy == 2 && !vy2)) continue;
        const int64_t row = nx * (sys[oy] + (int64_t)ny * szs[oz]);
        const int pyz = g.mx * (py[oy] + g.my * pz[oz]);
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
          if ((ox == 0 && !vx0) || (ox == 2 && !vx2)) continue;
          sum += corr[(sxs[ox] + row) * mxyz + px[ox] + pyz];
        }
      }
    }
    u[dof] = accumulate ? u[dof] + sum : sum;
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_scatter_n(const T* __restrict__ corr, T* __restrict__ u, int64_t Ne, int nx,
                                  int ny, int nz, SubShape g, int accumulate) {
  pdl_entry();
  scatter_n_body<T, N>(plain_block(), corr, u, Ne, nx, ny, nz, g, accumulate);
}

// k_scatter_n when every node lies in at most two subdomains per direction
// (2 N_O <= n): the two candidates of each direction in increasing offset,
// all eight loads issued unconditionally (an absent candidate repeats the own
// address and its value is replaced by zero), then summed in the same order
// as k_scatter_n, so the two kernels give identical bits.
template <typename T, int N>
__device__ __forceinline__ void scatter_n2_body(BlockIdx bi_, const T* __restrict__ corr, T* __restrict__ u,
                                                int64_t Ne, int nx, int ny, int nz, SubShape g, int accumulate) {
  constexpr int N3 = N * N * N;
  const int64_t mxyz = (int64_t)g.mx * g.my * g.mz;
  const int64_t total = Ne * N3;
  for (int64_t dof = bi_.b * (int64_t)blockDim.x + threadIdx.x; dof < total;
       dof += (int64_t)bi_.g * blockDim.x) {
    const int e = (int)(dof / N3);  // element indices fit in 32 bits
    const int loc = (int)(dof - (int64_t)e * N3);
    const int i = loc % N, j = (loc / N) % N, k = loc / (N * N);
    const int exy = e / nx;
    const int ex = e - exy * nx, ey = exy % ny, ez = exy / ny;
    int sx[2], px[2], sy[2], py[2], sz[2], pz[2];
    bool vx, vy, vz;
    auto cand = [&](int t, int no, int ec, int ne, int* sc, int* pc, bool* v) {
      if (t < no) {
        sc[0] = ec == 0 ? ne - 1 : ec - 1;
        pc[0] = no + N + t;
        sc[1] = ec;
        pc[1] = no + t;
        *v = true;
      } else if (t >= N - no) {
        sc[0] = ec;
        pc[0] = no + t;
        sc[1] = ec == ne - 1 ? 0 : ec + 1;
        pc[1] = t - (N - no);
        *v = true;
      } else {
        sc[0] = sc[1] = ec;
        pc[0] = pc[1] = no + t;
        *v = false;
      }
    };
    cand(i, g.nox, ex, nx, sx, px, &vx);
    cand(j, g.noy, ey, ny, sy, py, &vy);
    cand(k, g.noz, ez, nz, sz, pz, &vz);
    // offset of (subdomain, position) = the sum of one term per direction
    int64_t ox[2], oy[2], oz[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      ox[a] = sx[a] * mxyz + px[a];
      oy[a] = sy[a] * ((int64_t)nx * mxyz) + (int64_t)g.mx * py[a];
      oz[a] = sz[a] * ((int64_t)nx * ny * mxyz) + (int64_t)g.mx * g.my * pz[a];
    }
    T val[8];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) val[a + 2 * (b + 2 * c)] = corr[ox[a] + oy[b] + oz[c]];
    T sum = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a)
          if ((a == 0 || vx) && (b == 0 || vy) && (c == 0 || vz)) sum += val[a + 2 * (b + 2 * c)];
    u[dof] = accumulate ? u[dof] + sum : sum;
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_scatter_n2(const T* __restrict__ corr, T* __restrict__ u, int64_t Ne, int nx,
                                  int ny, int nz, SubShape g, int accumulate) {
  pdl_entry();
  scatter_n2_body<T, N>(plain_block(), corr, u, Ne, nx, ny, nz, g, accumulate);
}

// k_scatter_n2 with blocks aligned to elements: a block takes EPB whole
// elements (or, at high order, 1 / cpe of one element, so that a mesh of few
// elements still gives every SM blocks).  Per element and direction the two
// candidate contributions of every node position t -- the covering
// subdomains' share of the tile offset plus the position inside the tile --
// are formed once, in shared memory (cand[e][d][t][0..1]; a node covered by
// one subdomain only repeats its first candidate in the second); a DOF (i, j,
// k) then adds its <= 8 contributions cand_x[i][a] + cand_y[j][b] + cand_z[k][c]
// in the order of k_scatter_n / k_scatter_n2 (identical bits), with about a
// third of the per-DOF instructions of forming the candidates per DOF.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_scatter_e(const T* __restrict__ corr, T* __restrict__ u, int64_t Ne, int nx,
                                                   int ny, int nz, SubShape g, int accumulate, int cpe) {
  pdl_entry();
  constexpr int N3 = N * N * N, EPB = N3 >= 256 ? 1 : 256 / N3;
  __shared__ int64_t cand[EPB][3][N][2];
  const int64_t mxyz = (int64_t)g.mx * g.my * g.mz;
  const int tid = threadIdx.x, nt = blockDim.x;
  // work units: EPB elements, or (EPB = 1) the cpe chunks of an element
  const int chunk = EPB == 1 ? (N3 + cpe - 1) / cpe : N3;
  const int64_t units = EPB == 1 ? Ne * cpe : (Ne + EPB - 1) / EPB;
  for (int64_t vb = blockIdx.x; vb < units; vb += gridDim.x) {
    const int64_t e0 = EPB == 1 ? vb / cpe : vb * EPB;
    const int cnt = (int)(Ne - e0 < EPB ? Ne - e0 : EPB);
    const int d0 = EPB == 1 ? (int)(vb - e0 * cpe) * chunk : 0;
    const int d1 = EPB == 1 ? (d0 + chunk < N3 ? d0 + chunk : N3) : cnt * N3;
    for (int w = tid; w < cnt * 3 * N; w += nt) {
      const int ge = w / (3 * N), rem = w - ge * 3 * N, q = rem / N, t = rem - q * N;
      const int e = (int)(e0 + ge), exy = e / nx;  // element indices fit in 32 bits
      const int ex = e - exy * nx, ey = exy % ny, ez = exy / ny;
      const int no = q == 0 ? g.nox : (q == 1 ? g.noy : g.noz);
      const int ec = q == 0 ? ex : (q == 1 ? ey : ez), nd = q == 0 ? nx : (q == 1 ? ny : nz);
      const int64_t unit = q == 0 ? mxyz : (q == 1 ? (int64_t)nx * mxyz : (int64_t)nx * ny * mxyz);
      const int64_t pst = q == 0 ? 1 : (q == 1 ? (int64_t)g.mx : (int64_t)g.mx * g.my);
      // the two covering subdomains in increasing offset (or the own one twice)
      int oa0, pa0, oa1, pa1;
      if (t < no) {
        oa0 = -1; pa0 = no + N + t; oa1 = 0; pa1 = no + t;
      } else if (t >= N - no) {
        oa0 = 0; pa0 = no + t; oa1 = 1; pa1 = t - (N - no);
      } else {
        oa0 = oa1 = 0; pa0 = pa1 = no + t;
      }
      cand[ge][q][t][0] = wrap(ec + oa0, nd) * unit + pa0 * pst;
      cand[ge][q][t][1] = wrap(ec + oa1, nd) * unit + pa1 * pst;
    }
    __syncthreads();
    for (int d = d0 + tid; d < d1; d += nt) {
      const int ge = EPB == 1 ? 0 : d / N3;
      const int loc = EPB == 1 ? d : d - ge * N3;
      const int i = loc % N, j = (loc / N) % N, k = loc / (N * N);
      const int64_t x0 = cand[ge][0][i][0], x1 = cand[ge][0][i][1];
      const int64_t y0 = cand[ge][1][j][0], y1 = cand[ge][1][j][1];
      const int64_t z0 = cand[ge][2][k][0], z1 = cand[ge][2][k][1];
      const bool vx = x1 != x0, vy = y1 != y0, vz = z1 != z0;
      T sum = 0;
      if constexpr (!std::is_same<T, float>::value) {
        // FP64 and double-float: only the contributions that exist are loaded
        // and added (about 1.8 per node at N_O = 1 instead of eight: the FP64
        // pipe, or the dozen FP32 operations of a double-float add, bound the
        // masked form), in the same order
        sum += corr[x0 + y0 + z0];
        if (vx) sum += corr[x1 + y0 + z0];
        if (vy) {
          sum += corr[x0 + y1 + z0];
          if (vx) sum += corr[x1 + y1 + z0];
        }
        if (vz) {
          sum += corr[x0 + y0 + z1];
          if (vx) sum += corr[x1 + y0 + z1];
          if (vy) {
            sum += corr[x0 + y1 + z1];
            if (vx) sum += corr[x1 + y1 + z1];
          }
        }
      } else {
        // FP32: the eight loads issued together, the absent ones masked out
        // of the sum
        const bool v[3] = {vx, vy, vz};
        const int64_t ox[2] = {x0, x1}, oy[2] = {y0, y1}, oz[2] = {z0, z1};
        T val[8];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) val[a + 2 * (b + 2 * c)] = corr[ox[a] + oy[b] + oz[c]];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
              if ((a == 0 || v[0]) && (b == 0 || v[1]) && (c == 0 || v[2])) sum += val[a + 2 * (b + 2 * c)];
      }
      const int64_t dof = e0 * N3 + d;
      u[dof] = accumulate ? u[dof] + sum : sum;
    }
    __syncthreads();
  }
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
cudaError_t launch_fdm(const mg_ctx* c, int l, const T* r) {
  if (c->graded) {
    if constexpr (std::is_same<T, double>::value || std::is_same<T, float>::value)
      return launch_gfdm<T>(c, l, r);
    else
      return cudaErrorNotSupported;
  }
  const LevelInfo& lv = c->lev[l];
  if constexpr (std::is_same<T, float>::value) {
    if (lv.fdm_tc) {
      const cudaError_t e = launch_fdm_tc(c, l, r);
      if (e != cudaErrorNotSupported) return e;
    } else if (launch_recorder() == nullptr && (lv.fdm_variant != 1 || c->opts.fdm_operands)) {
      // single solves: the factors as kernel parameters (one kernel, or its
      // passes split over three, fdm_variant 2); batched solves keep the
      // shared-memory kernel, whose body has a grouped twin
      const cudaError_t e = launch_fdm_c(c, l, r);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  FdmArgs<T> a;
  a.tab = table_of<T>(c);
  a.r = r;
  a.corr = static_cast<T*>(c->ws.corr);
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.n = lv.n;
  a.m = lv.m[0];
  a.no = lv.no[0];
  for (int d = 0; d < 3; ++d) {
    a.md[d] = lv.m[d];
    a.nod[d] = lv.no[d];
    a.S[d] = lv.t[d].S;
    a.SW[d] = lv.t[d].SW;
  }
  a.dinv = lv.dinv;
  const bool cubic = lv.m[0] == lv.m[1] && lv.m[0] == lv.m[2];
  const int m = lv.m[0], m2 = m * m;
  if (cubic && (m & 1) && m >= 3 && m <= 35) {
    // compile-time width: several subdomains per block when m^2 is small
    const size_t smem = sizeof(T) * 6 * m2;
    // subdomains per block: FdmShape<T, m>::spb (the shared-memory tile is
    // sized for it), fewer for single solves on small meshes so that the
    // blocks still fill the SMs (batched records keep the fixed value: only
    // launches of equal shape merge)
    const int spb_max = m2 >= 100 ? 1 : 256 / m2;
    a.spb = launch_recorder() != nullptr
                ? spb_max
                : (int)std::max<int64_t>(1, std::min<int64_t>(spb_max, (c->Ne + 2 * 152 - 1) / (2 * 152)));
    a.s_in_smem = 1;
    int threads = a.spb * m2;
    threads = threads > 256 ? 256 : (threads + 31) / 32 * 32;
    int64_t groups = (c->Ne + a.spb - 1) / a.spb;
    int blocks = (int)(groups < 152 * 8 ? groups : 152 * 8);
    c->nlaunch += 1;
#define MGDG_CASE(M) case M: return launch_fdm_m<T, M>(a, blocks, threads, smem, c->stream);
    if constexpr (std::is_same<T, df64>::value) {
      switch (m) {
        MGDG_FDM_DF_WIDTHS(MGDG_CASE)
        default: break;
      }
    } else {
      switch (m) {
        MGDG_CASE(3) MGDG_CASE(5) MGDG_CASE(7) MGDG_CASE(9) MGDG_CASE(11) MGDG_CASE(13) MGDG_CASE(15)
        MGDG_CASE(17) MGDG_CASE(19) MGDG_CASE(21) MGDG_CASE(23) MGDG_CASE(25) MGDG_CASE(27) MGDG_CASE(29)
        MGDG_CASE(31) MGDG_CASE(33) MGDG_CASE(35)
        default: break;
      }
    }
#undef MGDG_CASE
    c->nlaunch -= 1;
  }
  a.spb = 1;
  size_t smem = 0;
  for (int d = 0; d < 3; ++d) smem += sizeof(T) * 2 * lv.m[d] * lv.m[d];
  a.s_in_smem = smem <= 160 * 1024;
  if (!a.s_in_smem) smem = 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fdm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int lines = std::max(lv.m[1] * lv.m[2], std::max(lv.m[0] * lv.m[2], lv.m[0] * lv.m[1]));
  int threads = lines >= 256 ? 256 : 128;
  int64_t blocks = c->Ne < 152 * 8 ? c->Ne : 152 * 8;
  launch_pdl<kTwinType<T> ? &fdm_body<T> : nullptr>(k_fdm<T>, (int)blocks, threads, smem, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter(const mg_ctx* c, int l, T* u, int accumulate) {
  const LevelInfo& lv = c->lev[l];
  int64_t total = lv.N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const T* corr = static_cast<const T*>(c->ws.corr);
  const int eb = (int)blocks;
  const SubShape g{lv.m[0], lv.m[1], lv.m[2], lv.no[0], lv.no[1], lv.no[2]};
  c->nlaunch += 1;
  const bool two = 2 * lv.no[0] <= lv.n && 2 * lv.no[1] <= lv.n && 2 * lv.no[2] <= lv.n;
  if (two && launch_recorder() == nullptr && !lv.scatter_plain) {
    // single solves: element-aligned blocks (batched solves keep k_scatter_n2, whose body has a twin)
    const int n3 = lv.n * lv.n * lv.n, epb = n3 >= 256 ? 1 : 256 / n3;
    // chunks per element (one-element blocks): at least 152 * 8 blocks in all where the
    // elements alone give fewer, each chunk at least 256 DOFs
    const int cpe = epb > 1 ? 1 : (int)std::max<int64_t>(1, std::min<int64_t>(n3 / 256, (152 * 8 + c->Ne - 1) / c->Ne));
    const int64_t eblocks = std::min<int64_t>(epb > 1 ? (c->Ne + epb - 1) / epb : c->Ne * cpe, 152 * 16);
    switch (lv.n) {
#define MGDG_SCE(N)                                                                                           \
  case N:                                                                                                     \
    launch_pdl(k_scatter_e<T, N>, (int)eblocks, 256, 0, c->stream, corr, u, c->Ne, c->ne[0], c->ne[1],        \
               c->ne[2], g, accumulate, cpe);                                                                 \
    return cudaGetLastError();
      MGDG_SCE(3) MGDG_SCE(5) MGDG_SCE(9) MGDG_SCE(17) MGDG_SCE(33)
#undef MGDG_SCE
      default: break;
    }
  }
  if (two) {
    switch (lv.n) {
#define MGDG_SC2(N)                                                                                           \
  case N:                                                                                                     \
    launch_pdl<kTwinType<T> ? &scatter_n2_body<T, N> : nullptr>(k_scatter_n2<T, N>, eb, 256, 0, c->stream, corr, u, \
                                                                c->Ne, c->ne[0], c->ne[1], c->ne[2], g,          \
                                                                accumulate);                                     \
    return cudaGetLastError();
      MGDG_SC2(3) MGDG_SC2(5) MGDG_SC2(9) MGDG_SC2(17) MGDG_SC2(33)
#undef MGDG_SC2
      default: break;
    }
  }
  switch (lv.n) {
#define MGDG_SC(N)                                                                                            \
  case N:                                                                                                     \
    launch_pdl<kTwinType<T> ? &scatter_n_body<T, N> : nullptr>(k_scatter_n<T, N>, eb, 256, 0, c->stream, corr, u,   \
                                                               c->Ne, c->ne[0], c->ne[1], c->ne[2], g,           \
                                                               accumulate);                                      \
    return cudaGetLastError();
    MGDG_SC(3) MGDG_SC(5) MGDG_SC(9) MGDG_SC(17) MGDG_SC(33)
#undef MGDG_SC
    default: break;
  }
  launch_pdl<kTwinType<T> ? &scatter_body<T> : nullptr>(k_scatter<T>, (int)blocks, 256, 0, c->stream, corr, u, c->Ne,
                                                        c->ne[0], c->ne[1], c->ne[2], lv.n, g, accumulate);
  return cudaGetLastError();
}

template cudaError_t launch_fdm<double>(const mg_ctx*, int, const double*);
template cudaError_t launch_fdm<float>(const mg_ctx*, int, const float*);
template cudaError_t launch_scatter<double>(const mg_ctx*, int, double*, int);
template cudaError_t launch_scatter<float>(const mg_ctx*, int, float*, int);
template cudaError_t launch_fdm<df64>(const mg_ctx*, int, const df64*);
template cudaError_t launch_scatter<df64>(const mg_ctx*, int, df64*, int);

}  // namespace mgdg
