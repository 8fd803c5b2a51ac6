"""Polynomial multigrid V-cycle, standalone MG and inexact preconditioned CG.

Section 3.2: levels P_l = 2^l, l = 0..L (P_0 = 1, P_L = P); A_l is the SIPG
matrix rediscretised with order P_l; the embedded interpolation I_l carries a
correction from level l-1 to level l, its transpose restricts residuals;
Algorithm 1 is the V-cycle with the weighted Schwarz smoother; the coarse
problem u_0 = A_0^+ f_0 is solved after projecting f_0 onto the range of A_0.
The Krylov acceleration is the inexact preconditioned CG of Golub and Ye with one
V-cycle as preconditioner.  Section 4 defines the convergence rate
rho = (r_n / r_0)^(1/n) with Euclidean residual norms.

Test infrastructure only (see ``oracle/__init__``).
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .gll import gll_nodes, lagrange_eval
from .schwarz import SchwarzSmoother, layer_delta, layers_from_width, max_layers, max_width_layers
from .sipg import assemble


def interpolation_matrix(P_coarse, P_fine):
    """Element matrix of the embedded interpolation (Section 3.2): the value of
    every coarse 3D basis function phi_i(x) phi_j(y) phi_k(z) (Eq. u_h, order
    P_coarse) at every fine GLL node (order P_fine); rows fine (a + n_f (b + n_f c)),
    columns coarse (i + n_c (j + n_c k))."""
    nf, nc = P_fine + 1, P_coarse + 1
    phi = lagrange_eval(gll_nodes(P_coarse), gll_nodes(P_fine))  # (nf, nc)
    I3 = np.zeros((nf ** 3, nc ** 3))
    for c in range(nf):
        for b in range(nf):
            for a in range(nf):
                row = a + nf * (b + nf * c)
                I3[row, :] = np.einsum("k,j,i->kji", phi[c], phi[b], phi[a]).ravel()
    return I3


def level_layers(P_l, n_o=None, delta_rel=None):
    """N_O on a level: prescribed layers clamped to floor(P_l/2)+1, or the layer
    count of a geometric width delta_O = delta_rel * dx (Table 1)."""
    if delta_rel is not None:
        return min(layers_from_width(P_l, delta_rel), max_layers(P_l))
    return min(int(n_o), max_layers(P_l))


def max_overlap_widths(mesh, frac):
    """The "max" overlap of Table 2: delta_O,i = min(max_j frac dx_j, dx_i), as a
    reference half-width 2 delta_O,i / dx_i per direction (<= 2)."""
    big = frac * max(mesh.h)
    return tuple(2.0 * min(big, mesh.h[d]) / mesh.h[d] for d in range(3))


class Level:
    def __init__(self, mesh, P_l, factor, n_o=None, delta_rel=None, smoother=True, profile="quintic",
                 max_frac=None, delta_rule=None):
        self.P = P_l
        self.A = assemble(mesh, P_l, factor)
        self.N = self.A.shape[0]
        self.smoother = None
        if smoother:
            if max_frac is not None:
                deltas = max_overlap_widths(mesh, max_frac)
                self.n_o = tuple(max_width_layers(P_l, d) for d in deltas)
                delta = deltas
            else:
                self.n_o = level_layers(P_l, n_o, delta_rel)
                # weight half-width: the strip itself for a geometric overlap,
                # else (or on request) a node-based reading (layer_delta)
                rule = delta_rule or ("strip" if delta_rel is not None else "mid")
                if rule == "strip":
                    if delta_rel is None:
                        raise ValueError("the strip reading needs a geometric overlap")
                    delta = min(2.0 * delta_rel, 1.0)
                else:
                    delta = layer_delta(P_l, self.n_o, rule)
            self.delta = delta
            self.smoother = SchwarzSmoother(self.A, mesh, P_l, self.n_o, delta, profile)


class Hierarchy:
    """All levels of the polynomial multigrid method for one mesh and order P."""

    def __init__(self, mesh, P, factor=2.0, n_o=1, delta_rel=None, profile="quintic", max_frac=None,
                 delta_rule=None):
        L = int(round(math.log2(P)))
        if 2 ** L != P:
            raise ValueError("P must be a power of two")
        self.mesh = mesh
        self.L = L
        self.levels = [Level(mesh, 2 ** l, factor, n_o, delta_rel, smoother=(l >= 1), profile=profile,
                             max_frac=max_frac, delta_rule=delta_rule) for l in range(L + 1)]
        self.I3 = [None] + [interpolation_matrix(2 ** (l - 1), 2 ** l) for l in range(1, L + 1)]
        self.Ne = mesh.num_elements

    @property
    def A(self):
        return self.levels[-1].A

    def prolong(self, l, uc):
        """I_l u_{l-1}: element-wise interpolation from level l-1 to level l."""
        I3 = self.I3[l]
        return (uc.reshape(self.Ne, I3.shape[1]) @ I3.T).ravel()

    def restrict(self, l, rf):
        """I_l^T r_l."""
        I3 = self.I3[l]
        return (rf.reshape(self.Ne, I3.shape[0]) @ I3).ravel()

    def coarse_solve(self, f0, dense_limit=4096):
        """u_0 = A_0^+ f_0.  f_0 is first projected onto the range of A_0,
        f_0 - mean(f_0) 1 (reading: the paper says 'null space'; the range is
        what makes the singular system solvable).  The minimum-norm solution is
        obtained directly: for N_0 <= dense_limit by a dense solve of
        (A_0 + 1 1^T / N_0) u = f_0, which equals A_0^+ f_0 for f_0 orthogonal to 1;
        otherwise by a sparse LU solve of (A_0 + e_0 e_0^T) v = f_0 (which forces
        v_0 = 0 and A_0 v = f_0) followed by removal of the mean of v."""
        A0 = self.levels[0].A
        f = f0 - f0.mean()
        N0 = len(f)
        if N0 <= dense_limit:
            u = np.linalg.solve(A0.toarray() + np.ones((N0, N0)) / N0, f)
        else:
            if getattr(self, "_coarse_lu", None) is None:
                pin = sp.csr_matrix(([1.0], ([0], [0])), shape=(N0, N0))
                self._coarse_lu = spl.splu((A0 + pin).tocsc())
            u = self._coarse_lu.solve(f)
        return u - u.mean()

    def smoother_steps(self, l, ns, growth):
        """N_s,l = ns * growth^(L - l) (growth 1: fixed V-cycle; 3: the variable
        V-cycle of Table 2)."""
        return ns * growth ** (self.L - l)

    def vcycle(self, u, f, ns1=1, ns2=1, growth=1):
        """Algorithm 1 (MultigridCycle) with the weighted Schwarz smoother."""
        L = self.L
        us = [None] * (L + 1)
        fs = [None] * (L + 1)
        us[L] = u.copy()
        fs[L] = f.copy()
        for l in range(L, 0, -1):
            lev = self.levels[l]
            if l < L:
                us[l] = np.zeros(lev.N)
            us[l] = lev.smoother.smooth(lev.A, us[l], fs[l], self.smoother_steps(l, ns1, growth))
            fs[l - 1] = self.restrict(l, fs[l] - lev.A @ us[l])
        us[0] = self.coarse_solve(fs[0])
        for l in range(1, L + 1):
            lev = self.levels[l]
            us[l] = us[l] + self.prolong(l, us[l - 1])
            us[l] = lev.smoother.smooth(lev.A, us[l], fs[l], self.smoother_steps(l, ns2, growth))
        return us[L]


def solve_mg(H, f, tol=1e-10, maxit=200, u0=None, ns1=1, ns2=1, growth=1):
    """Standalone MG: repeat V-cycles until ||f - A u||_2 <= tol ||f - A u_0||_2.
    Returns (u with zero Euclidean mean, cycles, residual-norm history)."""
    A = H.A
    u = np.zeros_like(f) if u0 is None else u0.copy()
    hist = [np.linalg.norm(f - A @ u)]
    it = 0
    while it < maxit:
        it += 1
        u = H.vcycle(u, f, ns1, ns2, growth)
        hist.append(np.linalg.norm(f - A @ u))
        if hist[-1] <= tol * hist[0]:
            break
    return u - u.mean(), it, hist


def solve_pcg(A, f, precond, tol=1e-10, maxit=200, x0=None):
    """Inexact preconditioned CG (Golub and Ye), the Krylov acceleration of
    Section 3.2, with beta_k = z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k).

    Reading (the algorithm is given only in an earlier reference): the residual
    and the preconditioned residual are projected to zero Euclidean mean in every
    iteration (the operator is singular with constant null space); convergence is
    tested on the recurrence residual against ||r_0||.
    Returns (x with zero mean, iterations, history of ||r_k||)."""
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - A @ x
    r = r - r.mean()
    hist = [np.linalg.norm(r)]
    z = precond(r)
    z = z - z.mean()
    p = z.copy()
    rz = np.dot(r, z)
    it = 0
    while it < maxit:
        it += 1
        q = A @ p
        alpha = rz / np.dot(p, q)
        x = x + alpha * p
        r_new = r - alpha * q
        r_new = r_new - r_new.mean()
        hist.append(np.linalg.norm(r_new))
        if hist[-1] <= tol * hist[0]:
            break
        z_new = precond(r_new)
        z_new = z_new - z_new.mean()
        beta = np.dot(z_new, r_new - r) / rz
        p = z_new + beta * p
        r, z = r_new, z_new
        rz = np.dot(r, z)
    return x - x.mean(), it, hist


def solve_mgcg(H, f, tol=1e-10, maxit=200, x0=None, ns1=1, ns2=1, growth=1):
    """MG-CG: inexact PCG preconditioned by one V-cycle from a zero guess."""
    return solve_pcg(H.A, f, lambda r: H.vcycle(np.zeros_like(r), r, ns1, ns2, growth),
                     tol=tol, maxit=maxit, x0=x0)


def convergence_rate(hist):
    """rho = (r_n / r_0)^(1/n) (Section 4) and rbar = -lg rho."""
    n = len(hist) - 1
    rho = (hist[-1] / hist[0]) ** (1.0 / n)
    return rho, -math.log10(rho)
