// Per-level 1D setup on the device (FP64), one thread block per level and
// direction.
//
// Section 2: GLL nodes, weights and differentiation matrix; 1D mass
// M = (h/2) diag(w) and SIPG stiffness L (element block K + face terms, face
// couplings to the neighbours), Eq. (A).
// Section 3.1: restricted 1D matrices L_s = R L R^T, M_s = R M R^T of the
// element-centred subdomain, the generalised eigenproblem L_s S = M_s S Lambda
// with S^T M_s S = I (solved as the symmetric problem
// M_s^{-1/2} L_s M_s^{-1/2} V = V Lambda, S = M_s^{-1/2} V), the hat weights w
// (Fig. wH), and the table 1/(lam_x + lam_y + lam_z) of the fast diagonalisation.
// Section 3.2: embedded interpolation J from order P_{l-1} to P_l; the
// eigenbasis of the whole periodic 1D problem on the coarsest level (used to
// apply A_0^+ directly).
//
// Both the subdomain problem and the periodic coarse problem are symmetric
// under reflection of the line, so the eigenproblem is split into its even and
// odd halves before the cyclic Jacobi iteration; every eigenvector is then
// exactly even or odd (the first ne columns of S are even, the rest odd).
#include <math.h>

#include "mg_internal.h"

namespace mgdg {
namespace {

constexpr int kSetupThreads = 256;
constexpr int kMaxSweeps = 60;

// Legendre polynomial L_P(x) and its first two derivatives (three-term
// recurrence; derivatives from (x^2-1) L_P' = P (x L_P - L_{P-1}) and the
// Legendre equation (1-x^2) L'' - 2x L' + P(P+1) L = 0), for |x| < 1.
__device__ void legendre(int P, double x, double* lp, double* dlp, double* d2lp) {
  double l0 = 1.0, l1 = x;
  for (int k = 1; k < P; ++k) {
    double l2 = ((2.0 * k + 1.0) * x * l1 - k * l0) / (k + 1.0);
    l0 = l1;
    l1 = l2;
  }
  *lp = l1;
  double d = P * (x * l1 - l0) / (x * x - 1.0);
  *dlp = d;
  *d2lp = (2.0 * x * d - P * (P + 1.0) * l1) / (1.0 - x * x);
}

__device__ double legendre_value(int P, double x) {
  if (P == 0) return 1.0;
  double l0 = 1.0, l1 = x;
  for (int k = 1; k < P; ++k) {
    double l2 = ((2.0 * k + 1.0) * x * l1 - k * l0) / (k + 1.0);
    l0 = l1;
    l1 = l2;
  }
  return l1;
}

// GLL nodes of order P by Newton's method on L_P'(x) = 0 from the
// Chebyshev-Gauss-Lobatto points, then symmetrised.  Single thread.
__device__ void gll_nodes_dev(int P, double* x) {
  const double pi = 3.14159265358979323846;
  x[0] = -1.0;
  x[P] = 1.0;
  for (int k = 1; k < P; ++k) {
    double t = -cos(pi * k / P);
    for (int it = 0; it < 100; ++it) {
      double lp, dlp, d2lp;
      legendre(P, t, &lp, &dlp, &d2lp);
      double dt = dlp / d2lp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[k] = t;
  }
  for (int k = 0; k <= P / 2; ++k) {
    double s = 0.5 * (x[P - k] - x[k]);
    x[k] = -s;
    x[P - k] = s;
  }
  if (P % 2 == 0) x[P / 2] = 0.0;
}

// Block-wide sum of one double per thread (kSetupThreads threads).
__device__ double block_sum(double v, double* sh) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// Cyclic Jacobi eigensolver for a symmetric n x n matrix A (row-major, global
// scratch), parallel round-robin ordering: n/2 disjoint rotations per step.
// On return the diagonal of A holds the eigenvalues and V (n x n) the
// eigenvectors as columns.  Returns false if kMaxSweeps sweeps did not bring
// the squared off-diagonal norm below tol2 times the squared diagonal norm
// (default 1e-30: 1e-15 of the norm).
__device__ bool jacobi(double* A, double* V, int n, double* sh_red, int* sh_p, int* sh_q, double* sh_c,
                       double* sh_s, double tol2 = 1e-30) {
  const int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < n * n; i += nt) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  if (n <= 1) return true;
  const int np = n + (n & 1);
  const int half = np / 2;
  bool converged = false;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = t; i < n * n; i += nt) {
      double v = A[i];
      if (i / n == i % n) dia += v * v; else off += v * v;
    }
    off = block_sum(off, sh_red);
    dia = block_sum(dia, sh_red);
    if (off <= tol2 * dia) {
      converged = true;
      break;
    }
    for (int round = 0; round < np - 1; ++round) {
      for (int k = t; k < half; k += nt) {
        int a = (k == 0) ? 0 : 1 + ((k - 1 + round) % (np - 1));
        int b = 1 + ((np - 2 - k + round) % (np - 1));
        int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = A[p * n + q];
          if (apq != 0.0) {
            double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        }
        sh_p[k] = p;
        sh_q[k] = q;
        sh_c[k] = c;
        sh_s[k] = s;
      }
      __syncthreads();
      for (int idx = t; idx < half * n; idx += nt) {  // rows: A <- J^T A
        int k = idx / n, j = idx % n;
        int p = sh_p[k], q = sh_q[k];
        if (q >= n) continue;
        double c = sh_c[k], s = sh_s[k];
        double apj = A[p * n + j], aqj = A[q * n + j];
        A[p * n + j] = c * apj - s * aqj;
        A[q * n + j] = s * apj + c * aqj;
      }
      __syncthreads();
      for (int idx = t; idx < half * n; idx += nt) {  // columns: A <- A J, V <- V J
        int k = idx / n, i = idx % n;
        int p = sh_p[k], q = sh_q[k];
        if (q >= n) continue;
        double c = sh_c[k], s = sh_s[k];
        double aip = A[i * n + p], aiq = A[i * n + q];
        A[i * n + p] = c * aip - s * aiq;
        A[i * n + q] = s * aip + c * aiq;
        double vip = V[i * n + p], viq = V[i * n + q];
        V[i * n + p] = c * vip - s * viq;
        V[i * n + q] = s * vip + c * viq;
      }
      __syncthreads();
    }
  }
  return converged;
}

// Symmetric generalised eigenproblem L S = M S Lambda (M diagonal > 0, L and M
// centro-symmetric, size m) by even/odd splitting and Jacobi.
// scratch: >= 4 m^2 doubles.  Writes S (m x m, column p = eigenvector p, even
// modes first) and lam (m).  Returns false on non-convergence.
__device__ bool gen_eig_centro(const double* L, const double* M, int m, double* S, double* lam, double* scratch,
                               double* sh_red, int* sh_p, int* sh_q, double* sh_c, double* sh_s) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int hm = m / 2, odd_m = m & 1;
  const int ne = hm + odd_m, no = hm;
  const double r2 = 0.70710678118654752440;
  double* E = scratch;
  double* VE = E + ne * ne;
  double* O = VE + ne * ne;
  double* VO = O + (no > 0 ? no * no : 1);
  // C = M^{-1/2} L M^{-1/2}
  auto C = [&](int a, int b) { return L[a * m + b] / sqrt(M[a] * M[b]); };
  for (int idx = t; idx < ne * ne; idx += nt) {
    int a = idx / ne, b = idx % ne;
    double v;
    if (a < hm && b < hm) v = C(a, b) + C(a, m - 1 - b);
    else if (a < hm) v = 2.0 * r2 * C(a, hm);
    else if (b < hm) v = 2.0 * r2 * C(hm, b);
    else v = C(hm, hm);
    E[idx] = v;
  }
  for (int idx = t; idx < no * no; idx += nt) {
    int a = idx / no, b = idx % no;
    O[idx] = C(a, b) - C(a, m - 1 - b);
  }
  __syncthreads();
  bool ok = jacobi(E, VE, ne, sh_red, sh_p, sh_q, sh_c, sh_s);
  ok = jacobi(O, VO, no, sh_red, sh_p, sh_q, sh_c, sh_s) && ok;
  for (int idx = t; idx < m * m; idx += nt) {
    int a = idx / m, p = idx % m;  // entry a of eigenvector p
    double v;
    if (p < ne) {
      int aa = a < hm ? a : (a >= m - hm ? m - 1 - a : hm);
      v = (aa < hm) ? VE[aa * ne + p] * r2 : VE[aa * ne + p];
    } else {
      int q = p - ne;
      if (a < hm) v = VO[a * no + q] * r2;
      else if (a >= m - hm) v = -VO[(m - 1 - a) * no + q] * r2;
      else v = 0.0;
    }
    S[idx] = v / sqrt(M[a]);
  }
  for (int p = t; p < m; p += nt) lam[p] = (p < ne) ? E[p * ne + p] : O[(p - ne) * no + (p - ne)];
  __syncthreads();
  return ok;
}

__device__ double quintic_step(double t) { return t * t * t * (10.0 - 15.0 * t + 6.0 * t * t); }

__device__ double hat_weight(double xi_h, double delta, int profile) {
  double a = fabs(xi_h);
  if (delta <= 0.0) return a < 1.0 ? 1.0 : (a == 1.0 ? 0.5 : 0.0);
  if (a <= 1.0 - delta) return 1.0;
  if (a >= 1.0 + delta) return 0.0;
  if (profile == MG_WEIGHT_QUINTIC_HALVES) {
    // a quintic step on each half of the strip, w = 1/2 on the interface
    return a <= 1.0 ? 1.0 - 0.5 * quintic_step((a - 1.0 + delta) / delta) : 0.5 * (1.0 - quintic_step((a - 1.0) / delta));
  }
  if (profile == MG_WEIGHT_QUINTIC_NORMALISED) {
    // one-sided hat r = 1 on the element, 1 - q((a - 1)/delta) in the strip,
    // normalised by the sum over the two subdomains covering the node
    const double d = fabs(a - 1.0);
    const double r = 1.0 - quintic_step(d / delta);
    return a <= 1.0 ? 1.0 / (1.0 + r) : r / (1.0 + r);
  }
  double tt = (a - 1.0 + delta) / (2.0 * delta);
  double q = (profile == MG_WEIGHT_LINEAR) ? tt : quintic_step(tt);
  return 1.0 - q;
}

struct SetupParams {
  int P, n, m, no, profile, level, Pc;
  double delta, h, g, mu;
  DirTables t;
  int64_t J;
  int Ng;        // coarse: 2 * elements in this direction
};

struct SetupBatch {
  SetupParams p[kMaxLevels * 3];
};

// Shared part of every block: GLL nodes/weights/D of order P in shared memory
// and the element block of L.
struct BasisSmem {
  double x[kMaxN], w[kMaxN], D[kMaxN * kMaxN], Lee[kMaxN * kMaxN];
  double xc[kMaxN], lamc[kMaxN];
  double red[kSetupThreads];
  int sp[kSetupThreads], sq[kSetupThreads];
  double sc[kSetupThreads], ss[kSetupThreads];
};

__device__ void build_basis(const SetupParams& q, BasisSmem& sm) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int P = q.P, n = q.n;
  if (t == 0) gll_nodes_dev(P, sm.x);
  __syncthreads();
  for (int i = t; i < n; i += nt) {
    double lp = legendre_value(P, sm.x[i]);
    sm.w[i] = 2.0 / (P * (P + 1.0) * lp * lp);
  }
  for (int idx = t; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    double v;
    if (i != j) v = legendre_value(P, sm.x[i]) / (legendre_value(P, sm.x[j]) * (sm.x[i] - sm.x[j]));
    else if (i == 0) v = -P * (P + 1.0) / 4.0;
    else if (i == P) v = P * (P + 1.0) / 4.0;
    else v = 0.0;
    sm.D[idx] = v;
  }
  __syncthreads();
  // element block: g D^T W D + mu (e_0 e_0^T + e_P e_P^T)
  //   - g/2 (e_P D_P + D_P^T e_P^T) + g/2 (e_0 D_0 + D_0^T e_0^T)
  const double g = q.g, mu = q.mu;
  for (int idx = t; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    double k = 0.0;
    for (int a = 0; a < n; ++a) k += sm.w[a] * sm.D[a * n + i] * sm.D[a * n + j];
    double v = g * k;
    if (i == j && (i == 0 || i == P)) v += mu;
    if (i == P) v -= 0.5 * g * sm.D[P * n + j];
    if (j == P) v -= 0.5 * g * sm.D[P * n + i];
    if (i == 0) v += 0.5 * g * sm.D[0 * n + j];
    if (j == 0) v += 0.5 * g * sm.D[0 * n + i];
    sm.Lee[idx] = v;
  }
  __syncthreads();
}

// 1D global-L entry between node i of element offset da and node j of element
// offset db (|da - db| <= 1, infinite or periodic line with >= 3 elements).
__device__ double line_entry(const BasisSmem& sm, const SetupParams& q, int da, int i, int db, int j) {
  const int n = q.n, P = q.P;
  const double g = q.g, mu = q.mu;
  if (da == db) return sm.Lee[i * n + j];
  if (db == da + 1) {  // row in the left element, column in the right one
    double v = 0.0;
    if (i == P && j == 0) v -= mu;
    if (i == P) v -= 0.5 * g * sm.D[0 * n + j];
    if (j == 0) v += 0.5 * g * sm.D[P * n + i];
    return v;
  }
  if (db == da - 1) {  // row in the right element, column in the left one
    double v = 0.0;
    if (i == 0 && j == P) v -= mu;
    if (i == 0) v += 0.5 * g * sm.D[P * n + j];
    if (j == P) v -= 0.5 * g * sm.D[0 * n + i];
    return v;
  }
  return 0.0;
}

__global__ void __launch_bounds__(kSetupThreads) k_setup_level(SetupBatch batch, double* tab, double* scratch,
                                  int64_t scratch_per_block, int* status) {
  __shared__ BasisSmem sm;
  const SetupParams q = batch.p[blockIdx.x];
  const int t = threadIdx.x, nt = blockDim.x;
  const int n = q.n;
  build_basis(q, sm);
  for (int i = t; i < n; i += nt) {
    tab[q.t.nodes + i] = sm.x[i];
    tab[q.t.weights + i] = sm.w[i];
    tab[q.t.mass + i] = 0.5 * q.h * sm.w[i];
    tab[q.t.d0 + i] = sm.D[0 * n + i];
    tab[q.t.dp + i] = sm.D[q.P * n + i];
  }
  for (int i = t; i < n * n; i += nt) tab[q.t.lee + i] = sm.Lee[i];
  // even/odd form of C = M^{-1} L_ee (centro-symmetric): for output i < ne
  //   (C u)_i = sum_{t<ne} ce[i][t] e_t + sum_{t<no} co[i][t] o_t,  (C u)_{n-1-i} = ... - ...
  // with e_t = u_t + u_{n-1-t}, o_t = u_t - u_{n-1-t} (t < no) and e_h = u_h for odd n.
  if (q.t.ce >= 0) {
    const int ne = (n + 1) / 2, no = n / 2;
    for (int idx = t; idx < ne * ne; idx += nt) {
      int i = idx / ne, tt = idx % ne;
      double mi = 0.5 * q.h * sm.w[i];
      double v = (tt < no) ? 0.5 * (sm.Lee[i * n + tt] + sm.Lee[i * n + n - 1 - tt]) : sm.Lee[i * n + tt];
      tab[q.t.ce + idx] = v / mi;
    }
    for (int idx = t; idx < no * no; idx += nt) {
      int i = idx / no, tt = idx % no;
      double mi = 0.5 * q.h * sm.w[i];
      tab[q.t.co + idx] = 0.5 * (sm.Lee[i * n + tt] - sm.Lee[i * n + n - 1 - tt]) / mi;
    }
    // face rank-1 terms -g/2 (D0_i a + D0_{n-1-i} c) in even/odd form (s = a + c, t = a - c)
    for (int i = t; i < ne; i += nt)
      tab[q.t.fe + i] = -0.25 * q.g * (sm.D[i] + sm.D[n - 1 - i]) / (0.5 * q.h * sm.w[i]);
    for (int i = t; i < no; i += nt)
      tab[q.t.fo + i] = -0.25 * q.g * (sm.D[i] - sm.D[n - 1 - i]) / (0.5 * q.h * sm.w[i]);
    if (t == 0) {
      double m0 = 0.5 * q.h * sm.w[0];
      tab[q.t.fsc + 0] = q.mu / m0;
      tab[q.t.fsc + 1] = 0.5 * q.g / m0;
    }
  }
  double* scr = scratch + blockIdx.x * scratch_per_block;

  if (q.level == 0) {
    // periodic coarse line of Ng = 2 * elements nodes, index 2 e + i
    const int Ng = q.Ng, ne = Ng / n;
    double* Lg = scr;
    double* Mg = Lg + Ng * Ng;
    double* wk = Mg + Ng;
    for (int idx = t; idx < Ng * Ng; idx += nt) {
      int r = idx / Ng, c = idx % Ng;
      int er = r / n, ir = r % n, ec = c / n, ic = c % n;
      int d = ec - er;
      if (d == ne - 1) d = -1;
      if (d == -(ne - 1)) d = 1;
      Lg[idx] = (d >= -1 && d <= 1) ? line_entry(sm, q, 0, ir, d, ic) : 0.0;
    }
    for (int i = t; i < Ng; i += nt) Mg[i] = 0.5 * q.h * sm.w[i % n];
    __syncthreads();
    bool ok = gen_eig_centro(Lg, Mg, Ng, tab + q.t.Q, tab + q.t.qlam, wk, sm.red, sm.sp, sm.sq, sm.sc, sm.ss);
    if (!ok && t == 0) atomicExch(status, kDevNoConv);
    return;
  }

  // element-centred subdomain line: last `no` nodes of the left neighbour, the
  // element, first `no` nodes of the right neighbour
  const int m = q.m, no = q.no;
  double* Ls = scr;
  double* Ms = Ls + m * m;
  double* wk = Ms + m;
  auto node_of = [&](int a, int* de, int* ii) {
    if (a < no) { *de = -1; *ii = n - no + a; }
    else if (a < no + n) { *de = 0; *ii = a - no; }
    else { *de = 1; *ii = a - no - n; }
  };
  for (int idx = t; idx < m * m; idx += nt) {
    int a = idx / m, b = idx % m, da, ia, db, ib;
    node_of(a, &da, &ia);
    node_of(b, &db, &ib);
    Ls[idx] = line_entry(sm, q, da, ia, db, ib);
  }
  for (int a = t; a < m; a += nt) {
    int da, ia;
    node_of(a, &da, &ia);
    Ms[a] = 0.5 * q.h * sm.w[ia];
    double xi_h = sm.x[ia] + 2.0 * da;
    double w = (no == 0) ? 1.0 : hat_weight(xi_h, q.delta, q.profile);
    if (no > 0 && q.delta > 1.0) {
      // A strip wider than half an element: the node of the neighbour element
      // may also lie in a third subdomain, so the weight is divided by the sum
      // of the raw weights of all subdomains covering it (xi_h - 2 o for the
      // subdomain centred o elements further on, o = -1, 0, +1).
      const double xi = sm.x[ia];
      double total = hat_weight(xi, q.delta, q.profile);
      if (ia >= n - no) total += hat_weight(xi - 2.0, q.delta, q.profile);
      if (ia < no) total += hat_weight(xi + 2.0, q.delta, q.profile);
      w = total > 0.0 ? w / total : 0.0;
    }
    tab[q.t.w + a] = w;
  }
  __syncthreads();
  bool ok = gen_eig_centro(Ls, Ms, m, tab + q.t.S, tab + q.t.lam, wk, sm.red, sm.sp, sm.sq, sm.sc, sm.ss);
  if (!ok && t == 0) atomicExch(status, kDevNoConv);
  __syncthreads();
  // S with the weights folded in: SW[a][p] = w[a] S[a][p]
  for (int idx = t; idx < m * m; idx += nt) tab[q.t.SW + idx] = tab[q.t.w + idx / m] * tab[q.t.S + idx];
  // interpolation from order Pc (barycentric form), written by the x block only
  if (q.J >= 0) {
    const int Pc = q.Pc, nc = Pc + 1;
    if (t == 0) gll_nodes_dev(Pc, sm.xc);
    __syncthreads();
    for (int i = t; i < nc; i += nt) {
      double prod = 1.0;
      for (int k = 0; k < nc; ++k)
        if (k != i) prod *= (sm.xc[i] - sm.xc[k]);
      sm.lamc[i] = 1.0 / prod;
    }
    __syncthreads();
    for (int idx = t; idx < n * nc; idx += nt) {
      int a = idx / nc, i = idx % nc;
      double xa = sm.x[a];
      int hit = -1;
      for (int k = 0; k < nc; ++k)
        if (fabs(xa - sm.xc[k]) < 1e-14) hit = k;
      double v;
      if (hit >= 0) {
        v = (hit == i) ? 1.0 : 0.0;
      } else {
        double den = 0.0;
        for (int k = 0; k < nc; ++k) den += sm.lamc[k] / (xa - sm.xc[k]);
        v = (sm.lamc[i] / (xa - sm.xc[i])) / den;
      }
      tab[q.J + idx] = v;
    }
  }
}

__global__ void k_setup_dinv(double* tab, int64_t dinv, int64_t lx, int64_t ly, int64_t lz, int mx, int my, int mz) {
  int64_t total = (int64_t)mx * my * mz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(i % mx), b = (int)((i / mx) % my), c = (int)(i / ((int64_t)mx * my));
    tab[dinv + i] = 1.0 / (tab[lx + a] + tab[ly + b] + tab[lz + c]);
  }
}

// 1 / (lam_x[a] + lam_y[b] + lam_z[c]) at (b + myp a) mzp + c, zero where b >= my or c >= mz.
__global__ void k_setup_dinvp(double* tab, int64_t dinvp, int64_t lx, int64_t ly, int64_t lz, int mx, int my, int mz) {
  const int myp = (my + 3) / 4 * 4, mzp = (mz + 3) / 4 * 4;
  const int64_t total = (int64_t)mx * myp * mzp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % mzp), row = (int)(i / mzp);
    const int b = row % myp, a = row / myp;
    tab[dinvp + i] = (b < my && c < mz) ? 1.0 / (tab[lx + a] + tab[ly + b] + tab[lz + c]) : 0.0;
  }
}

__global__ void k_setup_mass3(double* tab, int64_t mass3, int64_t mx, int64_t my, int64_t mz, int n) {
  const int total = n * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int a = i % n, b = (i / n) % n, c = i / (n * n);
    tab[mass3 + i] = tab[mx + a] * tab[my + b] * tab[mz + c];
  }
}

__global__ void k_cast_tables(const double* src, float* dst, df64* dst_df, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dst[i] = (float)src[i];
    dst_df[i] = df_from_double(src[i]);
  }
}

// ---- graded meshes: one eigenbasis per element line ----
//
// Element e of a line of widths h has the 1D matrix rows (Section 2, Eq. ip in
// one dimension, each element with its own g = 2/h, each face with the
// penalty of its smaller neighbour):
//   L[e][e]   = (2/h_e) K + mu_r e_P e_P^T - (1/h_e)(e_P D_P + D_P^T e_P^T)
//                         + mu_l e_0 e_0^T + (1/h_e)(e_0 D_0 + D_0^T e_0^T)
//   L[e][e+1] = -mu_r e_P e_0^T - (1/h_{e+1}) e_P D_0 + (1/h_e) D_P^T e_0^T
//   L[e][e-1] = -mu_l e_0 e_P^T + (1/h_{e-1}) e_0 D_P - (1/h_e) D_0^T e_P^T
// with K = D^T diag(w) D, D_0 / D_P the first / last row of D, mu_l / mu_r
// the penalties of the left / right face.  A subdomain line is not
// reflection-symmetric any more, so its generalised eigenproblem is solved
// whole (no even/odd split).

struct GradedLine {
  int level, dir, P, n, m, no, nd, first;  // first: index of the line's first block
  DirTables t;
  int64_t wid;                             // widths of the n_d elements (table offset)
  double pen;                              // penalty factor
};

struct GradedBatch {
  int count;                               // entries used
  GradedLine g[kMaxLevels * 3];
  int coarse_first;                        // first block of the three coarse blocks
  int Ng[3];
  DirTables tc[3];                         // level-0 tables (Q, qlam)
  int64_t wid[3];
  double pen;
};

// Entry (i, j) of the row block of an element of width h0 with neighbours of
// widths hm (left) and hp (right); column element offset db in {-1, 0, 1}.
__device__ double graded_entry(const double* D, const double* K, int n, double hm, double h0, double hp,
                               double mu_l, double mu_r, int db, int i, int j) {
  const int P = n - 1;
  double v = 0.0;
  if (db == 0) {
    v = (2.0 / h0) * K[i * n + j];
    if (i == P && j == P) v += mu_r;
    if (i == 0 && j == 0) v += mu_l;
    if (i == P) v -= D[P * n + j] / h0;
    if (j == P) v -= D[P * n + i] / h0;
    if (i == 0) v += D[0 * n + j] / h0;
    if (j == 0) v += D[0 * n + i] / h0;
  } else if (db == 1) {
    if (i == P && j == 0) v -= mu_r;
    if (i == P) v -= D[0 * n + j] / hp;
    if (j == 0) v += D[P * n + i] / h0;
  } else if (db == -1) {
    if (i == 0 && j == P) v -= mu_l;
    if (i == 0) v += D[P * n + j] / hm;
    if (j == P) v -= D[0 * n + i] / h0;
  }
  return v;
}

__device__ __forceinline__ double face_mu(double pen, int P, double a, double b) {
  return pen * P * (P + 1.0) / (2.0 * fmin(a, b));
}

// Symmetric generalised eigenproblem L S = M S Lambda (M diagonal > 0), the
// whole m x m problem by Jacobi.  C (m*m) holds L on entry and is overwritten;
// V: m*m scratch.  S[a][p] = entry a of eigenvector p, S^T M S = I.
__device__ bool gen_eig_full(double* C, const double* M, int m, double* V, double* S, double* lam, double* sh_red,
                             int* sh_p, int* sh_q, double* sh_c, double* sh_s) {
  const int t = threadIdx.x, nt = blockDim.x;
  for (int idx = t; idx < m * m; idx += nt) C[idx] /= sqrt(M[idx / m] * M[idx % m]);
  __syncthreads();
  // converged once the off-diagonal part is at the rounding level of an m x m
  // matrix: its norm at most 4 m eps of the diagonal's (the whole coarse line,
  // m up to 512, stalls above the fixed 1e-15 of the halved problems)
  const double eps = 2.220446049250313e-16;
  const double tol2 = fmax(1e-30, 16.0 * (double)m * m * eps * eps);
  const bool ok = jacobi(C, V, m, sh_red, sh_p, sh_q, sh_c, sh_s, tol2);
  for (int idx = t; idx < m * m; idx += nt) S[idx] = V[idx] / sqrt(M[idx / m]);
  for (int p = t; p < m; p += nt) lam[p] = C[p * m + p];
  __syncthreads();
  return ok;
}

struct GradedSmem {
  double x[kMaxN], w[kMaxN], D[kMaxN * kMaxN], K[kMaxN * kMaxN];
  double red[kSetupThreads];
  int sp[kSetupThreads], sq[kSetupThreads];
  double sc[kSetupThreads], ss[kSetupThreads];
};

__device__ void graded_basis(int P, GradedSmem& sm) {
  const int t = threadIdx.x, nt = blockDim.x, n = P + 1;
  if (t == 0) gll_nodes_dev(P, sm.x);
  __syncthreads();
  for (int i = t; i < n; i += nt) {
    const double lp = legendre_value(P, sm.x[i]);
    sm.w[i] = 2.0 / (P * (P + 1.0) * lp * lp);
  }
  for (int idx = t; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    double v;
    if (i != j) v = legendre_value(P, sm.x[i]) / (legendre_value(P, sm.x[j]) * (sm.x[i] - sm.x[j]));
    else if (i == 0) v = -P * (P + 1.0) / 4.0;
    else if (i == P) v = P * (P + 1.0) / 4.0;
    else v = 0.0;
    sm.D[idx] = v;
  }
  __syncthreads();
  for (int idx = t; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    double k = 0.0;
    for (int a = 0; a < n; ++a) k += sm.w[a] * sm.D[a * n + i] * sm.D[a * n + j];
    sm.K[idx] = k;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSetupThreads) k_setup_graded(GradedBatch b, double* tab, double* scratch,
                                                                int64_t per_line, int64_t per_coarse, int* status) {
  __shared__ GradedSmem sm;
  const int t = threadIdx.x, nt = blockDim.x;
  const int blk = blockIdx.x;
  if (blk >= b.coarse_first) {
    // periodic coarse line of the P = 1 level: Ng = 2 n_d nodes, index 2 e + i
    const int d = blk - b.coarse_first;
    const int Ng = b.Ng[d], nd = Ng / 2;
    graded_basis(1, sm);
    double* C = scratch + per_line * b.coarse_first + per_coarse * d;
    double* V = C + (int64_t)Ng * Ng;
    double* M = V + (int64_t)Ng * Ng;
    const double* h = tab + b.wid[d];
    for (int idx = t; idx < Ng * Ng; idx += nt) {
      const int r = idx / Ng, c = idx % Ng;
      const int er = r / 2, ir = r % 2, ec = c / 2, ic = c % 2;
      int db = ec - er;
      if (db == nd - 1) db = -1;
      if (db == -(nd - 1)) db = 1;
      double v = 0.0;
      if (db >= -1 && db <= 1) {
        const double hm = h[(er + nd - 1) % nd], h0 = h[er], hp = h[(er + 1) % nd];
        v = graded_entry(sm.D, sm.K, 2, hm, h0, hp, face_mu(b.pen, 1, hm, h0), face_mu(b.pen, 1, h0, hp), db, ir,
                         ic);
      }
      C[idx] = v;
    }
    for (int r = t; r < Ng; r += nt) M[r] = 0.5 * h[r / 2] * sm.w[r % 2];
    __syncthreads();
    const bool ok = gen_eig_full(C, M, Ng, V, tab + b.tc[d].Q, tab + b.tc[d].qlam, sm.red, sm.sp, sm.sq, sm.sc,
                                 sm.ss);
    if (!ok && t == 0) atomicExch(status, kDevNoConv);
    return;
  }
  int gi = 0;
  while (gi + 1 < b.count && blk >= b.g[gi + 1].first) ++gi;
  const GradedLine& g = b.g[gi];
  const int e = blk - g.first, nd = g.nd, n = g.n, P = g.P, m = g.m, no = g.no;
  graded_basis(P, sm);
  const double* h = tab + g.wid;
  // widths of the elements e-2 .. e+2 and the penalties of the four faces between them
  double hw[5], mu[4];
  for (int k = 0; k < 5; ++k) hw[k] = h[((e + k - 2) % nd + nd) % nd];
  for (int k = 0; k < 4; ++k) mu[k] = face_mu(g.pen, P, hw[k], hw[k + 1]);
  // rows of element e: L[e][e-1], L[e][e], L[e][e+1]; mass (h_e / 2) w
  double* blk3 = tab + g.t.gblk + (int64_t)e * 3 * n * n;
  for (int idx = t; idx < 3 * n * n; idx += nt) {
    const int db = idx / (n * n) - 1, i = (idx / n) % n, j = idx % n;
    blk3[idx] = graded_entry(sm.D, sm.K, n, hw[1], hw[2], hw[3], mu[1], mu[2], db, i, j);
  }
  for (int i = t; i < n; i += nt) tab[g.t.gmass + (int64_t)e * n + i] = 0.5 * hw[2] * sm.w[i];
  if (g.level == 0) return;
  // subdomain line centred on e: last `no` nodes of e-1, element e, first `no` nodes of e+1
  double* C = scratch + per_line * blk;
  double* V = C + (int64_t)m * m;
  double* M = V + (int64_t)m * m;
  auto node_of = [&](int a, int* de, int* ii) {
    if (a < no) { *de = -1; *ii = n - no + a; }
    else if (a < no + n) { *de = 0; *ii = a - no; }
    else { *de = 1; *ii = a - no - n; }
  };
  for (int idx = t; idx < m * m; idx += nt) {
    int a = idx / m, c = idx % m, da, ia, dc, ic;
    node_of(a, &da, &ia);
    node_of(c, &dc, &ic);
    // row element e + da: widths hw[1 + da .. 3 + da], faces mu[1 + da], mu[2 + da]
    C[idx] = graded_entry(sm.D, sm.K, n, hw[1 + da], hw[2 + da], hw[3 + da], mu[1 + da], mu[2 + da], dc - da, ia,
                          ic);
  }
  for (int a = t; a < m; a += nt) {
    int da, ia;
    node_of(a, &da, &ia);
    M[a] = 0.5 * hw[2 + da] * sm.w[ia];
  }
  __syncthreads();
  double* S = tab + g.t.gS + (int64_t)e * m * m;
  const bool ok = gen_eig_full(C, M, m, V, S, tab + g.t.glam + (int64_t)e * m, sm.red, sm.sp, sm.sq, sm.sc, sm.ss);
  if (!ok && t == 0) atomicExch(status, kDevNoConv);
  // weights in reference coordinates: the level's table w, folded into SW
  double* SW = tab + g.t.gSW + (int64_t)e * m * m;
  for (int idx = t; idx < m * m; idx += nt) SW[idx] = tab[g.t.w + idx / m] * S[idx];
}

}  // namespace

cudaError_t launch_setup_coarse_tables(const double len[3], const int ne[3], double penalty, double* tab,
                                       const DirTables t[3], double* scratch, int64_t per_block, int* status,
                                       cudaStream_t s) {
  SetupBatch batch;
  for (int d = 0; d < 3; ++d) {
    SetupParams& q = batch.p[d];
    q.P = 1;
    q.n = 2;
    q.m = 0;
    q.no = 0;
    q.profile = MG_WEIGHT_QUINTIC;
    q.level = 0;
    q.Pc = 0;
    q.delta = 0.0;
    q.h = len[d] / ne[d];
    q.g = 2.0 / q.h;
    q.mu = penalty * 2.0 / (2.0 * q.h);
    q.t = t[d];
    q.t.ce = q.t.co = q.t.fe = q.t.fo = q.t.fsc = -1;
    q.J = -1;
    q.Ng = 2 * ne[d];
  }
  k_setup_level<<<3, kSetupThreads, 0, s>>>(batch, tab, scratch, per_block, status);
  return cudaGetLastError();
}

cudaError_t launch_setup(mg_ctx* c) {
  SetupBatch batch;
  int nb = 0;
  for (int l = 0; l <= c->L; ++l) {
    const LevelInfo& lv = c->lev[l];
    for (int d = 0; d < 3; ++d) {
      SetupParams& q = batch.p[nb++];
      q.P = lv.P;
      q.n = lv.n;
      q.m = lv.m[d];
      q.no = lv.no[d];
      q.profile = c->opts.weight_profile;
      q.level = l;
      q.Pc = l > 0 ? c->lev[l - 1].P : 0;
      q.delta = lv.delta[d];
      q.h = lv.h[d];
      q.g = lv.g[d];
      q.mu = lv.mu[d];
      q.t = lv.t[d];
      q.J = (l > 0 && d == 0) ? lv.J : -1;
      q.Ng = (l == 0) ? c->Ng[d] : 0;
    }
  }
  int64_t per_block = c->ws.jac_count / nb;
  cudaStream_t s = c->stream;
  k_setup_level<<<nb, kSetupThreads, 0, s>>>(batch, c->ws.tab64, c->ws.jac, per_block, c->ws.status);
  c->nlaunch += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 0; l <= c->L; ++l) {
    const LevelInfo& lv = c->lev[l];
    if (lv.mass3 < 0) continue;
    int total = lv.n * lv.n * lv.n;
    k_setup_mass3<<<(total + 255) / 256, 256, 0, s>>>(c->ws.tab64, lv.mass3, lv.t[0].mass, lv.t[1].mass,
                                                      lv.t[2].mass, lv.n);
    c->nlaunch += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (int l = 1; l <= c->L; ++l) {
    const LevelInfo& lv = c->lev[l];
    int64_t total = (int64_t)lv.m[0] * lv.m[1] * lv.m[2];
    int blocks = (int)((total + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_setup_dinv<<<blocks, 256, 0, s>>>(c->ws.tab64, lv.dinv, lv.t[0].lam, lv.t[1].lam, lv.t[2].lam, lv.m[0],
                                        lv.m[1], lv.m[2]);
    k_setup_dinvp<<<blocks, 256, 0, s>>>(c->ws.tab64, lv.dinvp, lv.t[0].lam, lv.t[1].lam, lv.t[2].lam, lv.m[0],
                                         lv.m[1], lv.m[2]);
    c->nlaunch += 1;
    c->nlaunch += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (c->graded && (e = launch_setup_graded(c)) != cudaSuccess) return e;
  k_cast_tables<<<256, 256, 0, s>>>(c->ws.tab64, c->ws.tab32, c->ws.tabdf, c->ws.tab_count);
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_setup_graded(mg_ctx* c) {
  GradedBatch b;
  b.count = 0;
  int blocks = 0;
  for (int l = 0; l <= c->L; ++l) {
    const LevelInfo& lv = c->lev[l];
    for (int d = 0; d < 3; ++d) {
      GradedLine& g = b.g[b.count++];
      g.level = l;
      g.dir = d;
      g.P = lv.P;
      g.n = lv.n;
      g.m = lv.m[d];
      g.no = lv.no[d];
      g.nd = c->ne[d];
      g.first = blocks;
      g.t = lv.t[d];
      g.wid = c->gwid[d];
      g.pen = c->penalty;
      blocks += c->ne[d];
    }
  }
  b.coarse_first = blocks;
  for (int d = 0; d < 3; ++d) {
    b.Ng[d] = c->Ng[d];
    b.tc[d] = c->lev[0].t[d];
    b.wid[d] = c->gwid[d];
  }
  b.pen = c->penalty;
  k_setup_graded<<<blocks + 3, kSetupThreads, 0, c->stream>>>(b, c->ws.tab64, c->ws.gjac, c->ws.gjac_line,
                                                               c->ws.gjac_coarse, c->ws.status);
  c->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace mgdg
