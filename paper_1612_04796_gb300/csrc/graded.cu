// Level kernels for graded meshes: element widths varying along each axis of
// the periodic box (the mesh stays a tensor product, element (ex, ey, ez) is
// hx[ex] x hy[ey] x hz[ez]).  The paper's grids are uniform (Section 4); this
// file carries its operator (Section 2, Eq. A) and subdomain solves
// (Section 3.1) over to such meshes, where every element line has its own 1D
// matrix rows and every subdomain line its own eigenbasis.
//
// Operator (Eq. A with per-element factors): for node (i, j, k) of element e,
//   (A u)_ijk = sum_d (L_d u)_(line d) * m_d1 * m_d2,
// the 1D product along direction d using the rows of element e_d of L_d
// (blocks L[e][e-1], L[e][e], L[e][e+1] from the setup), the mass weights
// m = (h/2) w of the two other directions.  The coupling blocks are rank two
// (the face terms): L[e][e+1] has a full row P and otherwise only column 0,
// L[e][e-1] a full row 0 and otherwise only column P, so an interior row reads
// one value of each neighbour and a face row the neighbour's whole line.
//
// Smoother: the gather R_s r and the fast diagonalisation
//   du_s = (Sz (x) Sy (x) Sx) D^-1 (Sz^T (x) Sy^T (x) Sx^T) r_s,
// D = lam_x (+) lam_y (+) lam_z, with S, lam those of the subdomain lines
// through the subdomain's element and the weights folded into the backward
// factors; written to the correction buffer in the layout of the uniform
// smoother, so the uniform weighted scatter adds the corrections.
#include <algorithm>
#include <type_traits>

#include "mg_internal.h"

namespace mgdg {
namespace {

template <typename T>
const T* gtable(const mg_ctx* c);
template <>
const double* gtable<double>(const mg_ctx* c) { return c->ws.tab64; }
template <>
const float* gtable<float>(const mg_ctx* c) { return c->ws.tab32; }
template <>
const df64* gtable<df64>(const mg_ctx* c) { return c->ws.tabdf; }

__device__ __forceinline__ int gwrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

template <typename T>
struct GOpArgs {
  const T* tab;
  const T* u;
  const T* f;
  T* out;
  int64_t Ne;
  int nx, ny, nz, residual;
  int64_t blk[3], mass[3];
};

// One direction of the 1D product for node index i of the line through
// element e: line elements el (left), e, er (right); stride st between nodes
// of a line; base offsets of the three lines.
template <typename T, int N>
__device__ __forceinline__ T line_product(const T* __restrict__ B, const T* __restrict__ u, int64_t bl, int64_t bc,
                                          int64_t br, int st, int i) {
  constexpr int P = N - 1;
  const T* Bm = B;              // L[e][e-1]
  const T* B0 = B + N * N;      // L[e][e]
  const T* Bp = B + 2 * N * N;  // L[e][e+1]
  Acc<T> s;
  s.init(B0[i * N], u[bc]);
#pragma unroll
  for (int t = 1; t < N; ++t) s.add(B0[i * N + t], u[bc + t * st]);
  if (i == 0) {
#pragma unroll
    for (int t = 0; t < N; ++t) s.add(Bm[t], u[bl + t * st]);
  } else {
    s.add(Bm[i * N + P], u[bl + P * st]);
  }
  if (i == P) {
#pragma unroll
    for (int t = 0; t < N; ++t) s.add(Bp[P * N + t], u[br + t * st]);
  } else {
    s.add(Bp[i * N], u[br]);
  }
  return s.get();
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_gsipg(GOpArgs<T> a) {
  pdl_entry();
  constexpr int N3 = N * N * N;
  const int64_t total = a.Ne * N3;
  for (int64_t dof = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; dof < total;
       dof += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = dof / N3;
    const int loc = (int)(dof - e * N3);
    const int i = loc % N, j = (loc / N) % N, k = loc / (N * N);
    const int e32 = (int)e, exy = e32 / a.nx;
    const int ex = e32 - exy * a.nx, ey = exy % a.ny, ez = exy / a.ny;
    const T mx = a.tab[a.mass[0] + (int64_t)ex * N + i];
    const T my = a.tab[a.mass[1] + (int64_t)ey * N + j];
    const T mz = a.tab[a.mass[2] + (int64_t)ez * N + k];
    const int64_t rowy = (int64_t)a.nx * (ey + (int64_t)a.ny * ez);
    // x lines: nodes t + N (j + N k) of elements ex-1, ex, ex+1
    const int lx = N * (j + N * k);
    const T sx = line_product<T, N>(a.tab + a.blk[0] + (int64_t)ex * 3 * N * N, a.u,
                                    (gwrap(ex - 1, a.nx) + rowy) * N3 + lx, e * N3 + lx,
                                    (gwrap(ex + 1, a.nx) + rowy) * N3 + lx, 1, i);
    // y lines: nodes i + N (t + N k)
    const int ly = i + N * N * k;
    const int64_t ezrow = (int64_t)a.nx * a.ny * ez;
    const T sy = line_product<T, N>(a.tab + a.blk[1] + (int64_t)ey * 3 * N * N, a.u,
                                    (ex + (int64_t)a.nx * gwrap(ey - 1, a.ny) + ezrow) * N3 + ly, e * N3 + ly,
                                    (ex + (int64_t)a.nx * gwrap(ey + 1, a.ny) + ezrow) * N3 + ly, N, j);
    // z lines: nodes i + N j + N^2 t
    const int lz = i + N * j;
    const int64_t exy0 = ex + (int64_t)a.nx * ey, plane = (int64_t)a.nx * a.ny;
    const T sz = line_product<T, N>(a.tab + a.blk[2] + (int64_t)ez * 3 * N * N, a.u,
                                    (exy0 + plane * gwrap(ez - 1, a.nz)) * N3 + lz, e * N3 + lz,
                                    (exy0 + plane * gwrap(ez + 1, a.nz)) * N3 + lz, N * N, k);
    const T au = sx * my * mz + sy * mx * mz + sz * mx * my;
    a.out[dof] = a.residual ? a.f[dof] - au : au;
  }
}

// (Inner products through Acc<T>: a multiply-add chain in FP64 / FP32, the
// compensated double-float dot product for df64, the outer operator of the
// mixed solve with the outer iteration in double-float.)
// The same operator with each element staged in shared memory: one block per
// element (grid-stride), its n^3 values of u, the nine n x n row blocks of its
// three lines and its masses loaded once.  Phase A (every DOF, no branch):
// the diagonal-block products from shared memory plus, per direction and
// side, the coupling column that every row has (L[e][e-1] column P times the
// left neighbour's face value, L[e][e+1] column 0 times the right one's).
// Phases x, y, z: the rest of the two face rows of each direction (row 0 of
// L[e][e-1] and row P of L[e][e+1], the neighbour's whole line), one thread
// per face node, added to the face DOFs in shared memory (each phase touches
// every DOF at most once; a barrier between phases).  Splitting the face rows
// off keeps the warps of phase A from running the face loops of a few lanes.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_gsipg_s(GOpArgs<T> a) {
  pdl_entry();
  constexpr int N2 = N * N, N3 = N2 * N, P = N - 1;
  extern __shared__ __align__(16) unsigned char gs_raw[];
  T* su = reinterpret_cast<T*>(gs_raw);  // N^3
  T* sau = su + N3;                      // N^3: A u of the element
  T* sB = sau + N3;                      // [dir][block][N^2]: L[e][e-1], L[e][e], L[e][e+1]
  T* sm = sB + 9 * N2;                   // [dir][N]
  for (int64_t e = blockIdx.x; e < a.Ne; e += gridDim.x) {
    const int e32 = (int)e, exy = e32 / a.nx;
    const int ex = e32 - exy * a.nx, ey = exy % a.ny, ez = exy / a.ny;
    const int64_t bo[3] = {a.blk[0] + (int64_t)ex * 3 * N2, a.blk[1] + (int64_t)ey * 3 * N2,
                           a.blk[2] + (int64_t)ez * 3 * N2};
    const int64_t mo[3] = {a.mass[0] + (int64_t)ex * N, a.mass[1] + (int64_t)ey * N, a.mass[2] + (int64_t)ez * N};
    __syncthreads();  // the previous element's values are no longer read
    for (int q = threadIdx.x; q < N3; q += blockDim.x) su[q] = a.u[e * N3 + q];
    for (int q = threadIdx.x; q < 9 * N2; q += blockDim.x) {
      const int d = q / (3 * N2);
      sB[q] = a.tab[(d == 0 ? bo[0] : (d == 1 ? bo[1] : bo[2])) + (q - d * 3 * N2)];
    }
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
      const int d = q / N;
      sm[q] = a.tab[(d == 0 ? mo[0] : (d == 1 ? mo[1] : mo[2])) + (q - d * N)];
    }
    __syncthreads();
    const int64_t rowy = (int64_t)a.nx * (ey + (int64_t)a.ny * ez);
    const int64_t exl = (gwrap(ex - 1, a.nx) + rowy) * N3, exr = (gwrap(ex + 1, a.nx) + rowy) * N3;
    const int64_t ezrow = (int64_t)a.nx * a.ny * ez;
    const int64_t eyl = (ex + (int64_t)a.nx * gwrap(ey - 1, a.ny) + ezrow) * N3;
    const int64_t eyr = (ex + (int64_t)a.nx * gwrap(ey + 1, a.ny) + ezrow) * N3;
    const int64_t exy0 = ex + (int64_t)a.nx * ey, plane = (int64_t)a.nx * a.ny;
    const int64_t ezl = (exy0 + plane * gwrap(ez - 1, a.nz)) * N3, ezr = (exy0 + plane * gwrap(ez + 1, a.nz)) * N3;
    // phase A
    for (int q = threadIdx.x; q < N3; q += blockDim.x) {
      const int i = q % N, j = (q / N) % N, k = q / N2;
      T sx, sy, sz;
      {  // x lines: stride 1, base N (j + N k)
        const int b = N * (j + N * k);
        Acc<T> acc;
        acc.init(sB[N2 + i * N], su[b]);
#pragma unroll
        for (int t = 1; t < N; ++t) acc.add(sB[N2 + i * N + t], su[b + t]);
        acc.add(sB[i * N + P], a.u[exl + b + P]);
        acc.add(sB[2 * N2 + i * N], a.u[exr + b]);
        sx = acc.get();
      }
      {  // y lines: stride N, base i + N^2 k
        const int b = i + N2 * k;
        Acc<T> acc;
        acc.init(sB[4 * N2 + j * N], su[b]);
#pragma unroll
        for (int t = 1; t < N; ++t) acc.add(sB[4 * N2 + j * N + t], su[b + t * N]);
        acc.add(sB[3 * N2 + j * N + P], a.u[eyl + b + P * N]);
        acc.add(sB[5 * N2 + j * N], a.u[eyr + b]);
        sy = acc.get();
      }
      {  // z lines: stride N^2, base i + N j
        const int b = i + N * j;
        Acc<T> acc;
        acc.init(sB[7 * N2 + k * N], su[b]);
#pragma unroll
        for (int t = 1; t < N; ++t) acc.add(sB[7 * N2 + k * N + t], su[b + t * N2]);
        acc.add(sB[6 * N2 + k * N + P], a.u[ezl + b + P * N2]);
        acc.add(sB[8 * N2 + k * N], a.u[ezr + b]);
        sz = acc.get();
      }
      const T mx = sm[i], my = sm[N + j], mz = sm[2 * N + k];
      sau[q] = sx * my * mz + sy * mx * mz + sz * mx * my;
    }
    // phases x, y, z: face rows; task f < 2 N^2: side = f / N^2 (0: row 0 with the
    // left neighbour, 1: row P with the right one), (p, r) = the other two indices
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      __syncthreads();
      for (int f = threadIdx.x; f < 2 * N2; f += blockDim.x) {
        const int side = f / N2, pr = f - side * N2, p0 = pr % N, r0 = pr / N;
        const int st = d == 0 ? 1 : (d == 1 ? N : N2);
        // DOF of the face node and the base of its line
        const int base = d == 0 ? N * pr : (d == 1 ? p0 + N2 * r0 : pr);
        const int row = side == 0 ? 0 : P;
        const int64_t nb = d == 0 ? (side == 0 ? exl : exr) : (d == 1 ? (side == 0 ? eyl : eyr) : (side == 0 ? ezl : ezr));
        // L[e][e-1] row 0 without its column P, or L[e][e+1] row P without its column 0
        const T* B = sB + d * 3 * N2 + (side == 0 ? 0 : 2 * N2) + row * N;
        const int t0 = side == 0 ? 0 : 1;
        Acc<T> acc;
        acc.init(B[t0], a.u[nb + base + t0 * st]);
#pragma unroll
        for (int t = 1; t < N - 1; ++t) acc.add(B[t0 + t], a.u[nb + base + (t0 + t) * st]);
        // mass weights of the two other directions at the face node
        const T mo1 = d == 0 ? sm[N + p0] : sm[p0];
        const T mo2 = d == 2 ? sm[N + r0] : sm[2 * N + r0];
        const int q = base + row * st;
        sau[q] += acc.get() * mo1 * mo2;
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < N3; q += blockDim.x) {
      const int64_t dof = e * N3 + q;
      a.out[dof] = a.residual ? a.f[dof] - sau[q] : sau[q];
    }
  }
}

template <typename T, int N>
cudaError_t launch_gsipg_s(const mg_ctx* c, const GOpArgs<T>& a) {
  constexpr size_t smem = sizeof(T) * (2 * N * N * N + 9 * N * N + 3 * N);
  static std::atomic<size_t> smem_set{48 * 1024};
  const cudaError_t e = allow_smem((const void*)k_gsipg_s<T, N>, smem, smem_set);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<int64_t>(a.Ne, 152 * 8);
  launch_pdl(k_gsipg_s<T, N>, blocks, 256, smem, c->stream, a);
  return cudaGetLastError();
}

template <typename T>
struct GFdmArgs {
  const T* tab;
  const T* r;
  T* corr;
  int64_t Ne;
  int nx, ny, nz, n;
  int md[3], nod[3];
  int64_t S[3], SW[3], lam[3];
};

__device__ __forceinline__ void gsub_node(int a, int n, int no, int* de, int* ii) {
  if (a < no) { *de = -1; *ii = n - no + a; }
  else if (a < no + n) { *de = 0; *ii = a - no; }
  else { *de = 1; *ii = a - no - n; }
}

// Shared memory: S and SW of the three directions (2 m_d^2 each) and lam
// (m_d each) of the subdomain being transformed.
template <typename T>
__global__ void __launch_bounds__(256) k_gfdm(GFdmArgs<T> a) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  T* sm = reinterpret_cast<T*>(gsm_raw);
  const int mx = a.md[0], my = a.md[1], mz = a.md[2], mxy = mx * my, mxyz = mxy * mz;
  const int n = a.n, n3 = n * n * n, nox = a.nod[0], noy = a.nod[1], noz = a.nod[2];
  T* S[3];
  T* SW[3];
  T* lam[3];
  {
    T* p = sm;
    for (int d = 0; d < 3; ++d) {
      S[d] = p;
      SW[d] = p + a.md[d] * a.md[d];
      p += 2 * a.md[d] * a.md[d];
    }
    for (int d = 0; d < 3; ++d) {
      lam[d] = p;
      p += a.md[d];
    }
  }
  T x[kMaxM], v[kMaxM];
  for (int64_t s = blockIdx.x; s < a.Ne; s += gridDim.x) {
    const int s32 = (int)s, sxy = s32 / a.nx;
    const int sx = s32 - sxy * a.nx, sy = sxy % a.ny, sz = sxy / a.ny;
    const int line[3] = {sx, sy, sz};
    __syncthreads();  // the previous subdomain's factors are no longer read
    for (int d = 0; d < 3; ++d) {
      const int m2 = a.md[d] * a.md[d];
      const T* gS = a.tab + a.S[d] + (int64_t)line[d] * m2;
      const T* gSW = a.tab + a.SW[d] + (int64_t)line[d] * m2;
      for (int q = threadIdx.x; q < m2; q += blockDim.x) {
        S[d][q] = gS[q];
        SW[d][q] = gSW[q];
      }
      const T* gl = a.tab + a.lam[d] + (int64_t)line[d] * a.md[d];
      for (int q = threadIdx.x; q < a.md[d]; q += blockDim.x) lam[d][q] = gl[q];
    }
    __syncthreads();
    T* tile = a.corr + s * (int64_t)mxyz;
    const int64_t exl = gwrap(sx - 1, a.nx), exr = gwrap(sx + 1, a.nx);
    // pass 1: gather the x-lines of r_s = R_s r, forward transform along x
    for (int ln = threadIdx.x; ln < my * mz; ln += blockDim.x) {
      const int b = ln % my, c = ln / my;
      int dy, iy, dz, iz;
      gsub_node(b, n, noy, &dy, &iy);
      gsub_node(c, n, noz, &dz, &iz);
      const int64_t row = a.nx * (gwrap(sy + dy, a.ny) + (int64_t)a.ny * gwrap(sz + dz, a.nz));
      const int loc = n * (iy + n * iz);
      const T* rl = a.r + (exl + row) * n3 + loc;
      const T* rc = a.r + (sx + row) * n3 + loc;
      const T* rr = a.r + (exr + row) * n3 + loc;
      for (int t = 0; t < nox; ++t) x[t] = rl[n - nox + t];
      for (int t = 0; t < n; ++t) x[nox + t] = rc[t];
      for (int t = 0; t < nox; ++t) x[nox + n + t] = rr[t];
      T* out = tile + mx * ln;
      for (int p = 0; p < mx; ++p) {
        T acc = 0;
        for (int q = 0; q < mx; ++q) acc += S[0][q * mx + p] * x[q];
        out[p] = acc;
      }
    }
    __syncthreads();
    // pass 2: forward along y
    for (int ln = threadIdx.x; ln < mx * mz; ln += blockDim.x) {
      T* lp = tile + (ln % mx) + mxy * (ln / mx);
      for (int t = 0; t < my; ++t) x[t] = lp[t * mx];
      for (int p = 0; p < my; ++p) {
        T acc = 0;
        for (int q = 0; q < my; ++q) acc += S[1][q * my + p] * x[q];
        lp[p * mx] = acc;
      }
    }
    __syncthreads();
    // pass 3: forward along z, divide by lam_x + lam_y + lam_z, backward along z
    for (int ln = threadIdx.x; ln < mxy; ln += blockDim.x) {
      T* lp = tile + ln;
      const T lxy = lam[0][ln % mx] + lam[1][ln / mx];
      for (int t = 0; t < mz; ++t) x[t] = lp[t * mxy];
      for (int p = 0; p < mz; ++p) {
        T acc = 0;
        for (int q = 0; q < mz; ++q) acc += S[2][q * mz + p] * x[q];
        v[p] = acc / (lxy + lam[2][p]);
      }
      for (int q = 0; q < mz; ++q) {
        T acc = 0;
        for (int p = 0; p < mz; ++p) acc += SW[2][q * mz + p] * v[p];
        lp[q * mxy] = acc;
      }
    }
    __syncthreads();
    // pass 4: backward along y
    for (int ln = threadIdx.x; ln < mx * mz; ln += blockDim.x) {
      T* lp = tile + (ln % mx) + mxy * (ln / mx);
      for (int t = 0; t < my; ++t) v[t] = lp[t * mx];
      for (int q = 0; q < my; ++q) {
        T acc = 0;
        for (int p = 0; p < my; ++p) acc += SW[1][q * my + p] * v[p];
        lp[q * mx] = acc;
      }
    }
    __syncthreads();
    // pass 5: backward along x (weights folded into SW)
    for (int ln = threadIdx.x; ln < my * mz; ln += blockDim.x) {
      T* lp = tile + mx * ln;
      for (int t = 0; t < mx; ++t) v[t] = lp[t];
      for (int q = 0; q < mx; ++q) {
        T acc = 0;
        for (int p = 0; p < mx; ++p) acc += SW[0][q * mx + p] * v[p];
        lp[q] = acc;
      }
    }
  }
}

// Mean removal on level 0 in two launches: per-block partial sums of x into
// red[0 .. nb), then out = x - (sum of the partials, in block order) / n,
// every block adding the nb partials itself.
template <typename T>
__global__ void __launch_bounds__(256) k_gsum_partial(const T* __restrict__ x, int64_t n, double* __restrict__ red) {
  pdl_entry();
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) red[blockIdx.x] = sh[0];
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_gsub_mean(const TI* x, TO* out, int64_t n, const double* __restrict__ red,
                                                   int nb) {
  pdl_entry();
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nb; ++q) s += red[q];
    mean = s / (double)n;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)((double)x[i] - mean);
}

struct GMassArgs {
  const double* tab;
  int64_t mass[3];
  int n, nx, ny;
  int64_t Ne;
};

__device__ __forceinline__ double gmass_at(const GMassArgs& a, int64_t dof) {
  const int n = a.n, n3 = n * n * n;
  const int64_t e = dof / n3;
  const int loc = (int)(dof - e * n3);
  const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
  const int64_t ex = e % a.nx, ey = (e / a.nx) % a.ny, ez = e / ((int64_t)a.nx * a.ny);
  return a.tab[a.mass[0] + ex * n + i] * a.tab[a.mass[1] + ey * n + j] * a.tab[a.mass[2] + ez * n + k];
}

// Per-block partial sums of M f (red[b]) and of M (red[nb + b]).
__global__ void __launch_bounds__(256) k_gmass_partial(GMassArgs a, const double* __restrict__ f, double* red) {
  pdl_entry();
  __shared__ double s0[256], s1[256];
  const int64_t total = a.Ne * a.n * a.n * a.n;
  double p0 = 0.0, p1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double m = gmass_at(a, i);
    p0 += m * f[i];
    p1 += m;
  }
  s0[threadIdx.x] = p0;
  s1[threadIdx.x] = p1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    red[blockIdx.x] = s0[0];
    red[gridDim.x + blockIdx.x] = s1[0];
  }
}

// b = M (f - fbar), fbar = (sum M f) / (sum M) from the partial sums.
__global__ void __launch_bounds__(256) k_grhs(GMassArgs a, const double* __restrict__ f, double* __restrict__ b,
                                              const double* __restrict__ red, int nb) {
  pdl_entry();
  __shared__ double fbar;
  if (threadIdx.x == 0) {
    double mf = 0.0, mm = 0.0;
    for (int q = 0; q < nb; ++q) {
      mf += red[q];
      mm += red[nb + q];
    }
    fbar = mf / mm;
  }
  __syncthreads();
  const int64_t total = a.Ne * a.n * a.n * a.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = gmass_at(a, i) * (f[i] - fbar);
}

__global__ void __launch_bounds__(256) k_gcoords(const double* tab, int64_t nodes, int n, int64_t Ne, int nx, int ny,
                                                 int64_t w0, int64_t w1, int64_t w2, int64_t o0, int64_t o1,
                                                 int64_t o2, double* x, double* y, double* z) {
  pdl_entry();
  const int n3 = n * n * n;
  const int64_t total = Ne * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / n3;
    const int loc = (int)(idx - e * n3);
    const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    x[idx] = tab[o0 + ex] + (tab[nodes + i] + 1.0) * 0.5 * tab[w0 + ex];
    y[idx] = tab[o1 + ey] + (tab[nodes + j] + 1.0) * 0.5 * tab[w1 + ey];
    z[idx] = tab[o2 + ez] + (tab[nodes + k] + 1.0) * 0.5 * tab[w2 + ez];
  }
}

inline int ggrid(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

}  // namespace

template <typename T>
cudaError_t launch_gsipg(const mg_ctx* c, int l, const T* u, const T* f, T* out, int residual) {
  const LevelInfo& lv = c->lev[l];
  GOpArgs<T> a;
  a.tab = gtable<T>(c);
  a.u = u;
  a.f = f;
  a.out = out;
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.residual = residual;
  for (int d = 0; d < 3; ++d) {
    a.blk[d] = lv.t[d].gblk;
    a.mass[d] = lv.t[d].gmass;
  }
  const int blocks = ggrid(lv.N, 256);
  c->nlaunch += 1;
  switch (lv.n) {
    case 5: return launch_gsipg_s<T, 5>(c, a);
    case 9: return launch_gsipg_s<T, 9>(c, a);
    case 17: return launch_gsipg_s<T, 17>(c, a);
    default: break;
  }
  switch (lv.n) {
    case 2: launch_pdl(k_gsipg<T, 2>, blocks, 256, 0, c->stream, a); break;
    case 3: launch_pdl(k_gsipg<T, 3>, blocks, 256, 0, c->stream, a); break;
    case 5: launch_pdl(k_gsipg<T, 5>, blocks, 256, 0, c->stream, a); break;
    case 9: launch_pdl(k_gsipg<T, 9>, blocks, 256, 0, c->stream, a); break;
    case 17: launch_pdl(k_gsipg<T, 17>, blocks, 256, 0, c->stream, a); break;
    case 33: launch_pdl(k_gsipg<T, 33>, blocks, 256, 0, c->stream, a); break;
    default: c->nlaunch -= 1; return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gfdm(const mg_ctx* c, int l, const T* r) {
  const cudaError_t ef = launch_gfdm_fixed<T>(c, l, r);
  if (ef != cudaErrorNotSupported) return ef;
  const LevelInfo& lv = c->lev[l];
  GFdmArgs<T> a;
  a.tab = gtable<T>(c);
  a.r = r;
  a.corr = static_cast<T*>(c->ws.corr);
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.n = lv.n;
  size_t smem = 0;
  for (int d = 0; d < 3; ++d) {
    a.md[d] = lv.m[d];
    a.nod[d] = lv.no[d];
    a.S[d] = lv.t[d].gS;
    a.SW[d] = lv.t[d].gSW;
    a.lam[d] = lv.t[d].glam;
    smem += sizeof(T) * (2 * (size_t)lv.m[d] * lv.m[d] + lv.m[d]);
  }
  static std::atomic<size_t> smem_set_d{48 * 1024}, smem_set_f{48 * 1024};
  cudaError_t e = allow_smem((const void*)k_gfdm<T>, smem,
                             std::is_same<T, double>::value ? smem_set_d : smem_set_f);
  if (e != cudaSuccess) return e;
  const int lines = std::max(lv.m[1] * lv.m[2], std::max(lv.m[0] * lv.m[2], lv.m[0] * lv.m[1]));
  const int threads = lines >= 256 ? 256 : (lines + 31) / 32 * 32;
  const int blocks = (int)std::min<int64_t>(c->Ne, 152 * 8);
  launch_pdl(k_gfdm<T>, blocks, threads, smem, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// Blocks of the level-0 mean removals: about 2,048 values per block, at most 64.
inline int gmean_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, (n + 2047) / 2048)); }

template <typename T>
cudaError_t launch_gmean_zero(const mg_ctx* c, T* u0) {
  const int64_t n = c->lev[0].N;
  const int nb = gmean_blocks(n);
  launch_pdl(k_gsum_partial<T>, nb, 256, 0, c->stream, (const T*)u0, n, c->ws.red);
  launch_pdl(k_gsub_mean<T, T>, nb, 256, 0, c->stream, (const T*)u0, u0, n, (const double*)c->ws.red, nb);
  c->nlaunch += 2;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gcenter(const mg_ctx* c, const T* f0, double* out) {
  const int64_t n = c->lev[0].N;
  const int nb = gmean_blocks(n);
  launch_pdl(k_gsum_partial<T>, nb, 256, 0, c->stream, f0, n, c->ws.red);
  launch_pdl(k_gsub_mean<T, double>, nb, 256, 0, c->stream, f0, out, n, (const double*)c->ws.red, nb);
  c->nlaunch += 2;
  return cudaGetLastError();
}

cudaError_t launch_grhs(const mg_ctx* c, const double* f, double* b) {
  const LevelInfo& lv = c->lev[c->L];
  GMassArgs a;
  a.tab = c->ws.tab64;
  for (int d = 0; d < 3; ++d) a.mass[d] = lv.t[d].gmass;
  a.n = lv.n;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.Ne = c->Ne;
  const int nb = reduction_blocks(lv.N);
  launch_pdl(k_gmass_partial, nb, 256, 0, c->stream, a, f, c->ws.red);
  launch_pdl(k_grhs, ggrid(lv.N, 256), 256, 0, c->stream, a, f, b, (const double*)c->ws.red, nb);
  c->nlaunch += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_sum(c, b, lv.N, kSlotSum)) != cudaSuccess) return e;
  return launch_sub_mean(c, b, lv.N, kSlotSum);
}

cudaError_t launch_gcoords(const mg_ctx* c, int l, double* x, double* y, double* z) {
  const LevelInfo& lv = c->lev[l];
  launch_pdl(k_gcoords, ggrid(lv.N, 256), 256, 0, c->stream, (const double*)c->ws.tab64, lv.t[0].nodes, lv.n,
             c->Ne, c->ne[0], c->ne[1], c->gwid[0], c->gwid[1], c->gwid[2], c->gorg[0], c->gorg[1], c->gorg[2], x, y,
             z);
  c->nlaunch += 1;
  return cudaGetLastError();
}

template cudaError_t launch_gsipg<double>(const mg_ctx*, int, const double*, const double*, double*, int);
template cudaError_t launch_gsipg<float>(const mg_ctx*, int, const float*, const float*, float*, int);
template cudaError_t launch_gsipg<df64>(const mg_ctx*, int, const df64*, const df64*, df64*, int);
template cudaError_t launch_gfdm<double>(const mg_ctx*, int, const double*);
template cudaError_t launch_gfdm<float>(const mg_ctx*, int, const float*);
template cudaError_t launch_gmean_zero<double>(const mg_ctx*, double*);
template cudaError_t launch_gmean_zero<float>(const mg_ctx*, float*);
template cudaError_t launch_gcenter<double>(const mg_ctx*, const double*, double*);
template cudaError_t launch_gcenter<float>(const mg_ctx*, const float*, double*);

}  // namespace mgdg
