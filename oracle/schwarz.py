"""Weighted overlapping additive Schwarz smoother on element-centred subdomains.

Section 3.1: each subdomain Omega_s is element s plus an overlap strip adopted
from the surrounding elements (N_O node layers, or a width delta_O).  With the
restriction R_s, the local problem is A_ss du_s = r_s, A_ss = R_s A R_s^T,
r_s = R_s r (Eq. subproblem); one additive Schwarz step adds
sum_s R_s^T (W_s du_s) (Eq. correction:global), W_s = W_z (x) W_y (x) W_x built
from the hat-shaped weight function w_H (Fig. wH).

This oracle solves each A_ss DIRECTLY (dense Cholesky, or sparse LU for large
subdomains), i.e. it does not use the fast diagonalisation the method uses; the
two agree up to rounding because fast diagonalisation is an exact
factorisation of A_ss^{-1}.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .gll import gll_nodes


def max_width_layers(P, delta_ref):
    """N_O for a strip of reference half-width delta_ref that may reach the
    whole neighbour element (delta_ref <= 2): all neighbour nodes within it."""
    xi = gll_nodes(P)
    return int(np.sum(1.0 + xi <= delta_ref + 1e-12))


def max_layers(P):
    """Largest admissible N_O at order P: floor(P/2) + 1, the layer count of
    delta_O = dx/2, the widest overlap the paper uses (Table 1, rows 5-6).

    Reading: the paper states the limit only geometrically (delta_O may not
    exceed the width of the adjoining element, Section 3.1); a node may lie in at
    most two subdomains per direction for the weights to sum to one, so N_O is
    clamped to this value on every level."""
    return P // 2 + 1


def layers_from_width(P, delta_rel):
    """N_O for a geometric overlap delta_O = delta_rel * dx: the number of
    neighbour GLL nodes whose distance from the interface is <= delta_O.

    In reference units the distance of neighbour node k is 1 + xi_k and the
    overlap half-width is 2 delta_O / dx.  Inclusive comparison (a node exactly on
    the strip boundary counts) reproduces the GLL N_O column of Table 1."""
    xi = gll_nodes(P)
    return int(np.sum(1.0 + xi <= 2.0 * delta_rel + 1e-12))


def quintic(t):
    """q(t) = 10 t^3 - 15 t^4 + 6 t^5: the quintic transition from 0 to 1 with
    q(t) + q(1-t) = 1 (reading of 'piece-wise quintic transition', Fig. wH)."""
    return t ** 3 * (10.0 - 15.0 * t + 6.0 * t ** 2)


def hat_weight(xi_h, delta, profile="quintic"):
    """w_H(xi_H) for overlap half-width ``delta`` in reference units (Fig. wH).

    Reading (the full definition is deferred to an earlier paper): w = 1 for
    |xi_H| <= 1 - delta, w = 0 for |xi_H| >= 1 + delta, and
    w = 1 - q((|xi_H| - 1 + delta) / (2 delta)) in between, so w = 1/2 on the
    interface and neighbouring subdomains' weights sum to one.  ``profile``
    selects q: "quintic" (the paper's wording) or "linear" (q(t) = t); or one of
    two other readings of a "piece-wise quintic transition": "quintic_halves"
    (a quintic step on each half of the strip) and "quintic_normalised" (a
    one-sided quintic hat normalised to a partition of unity).  All give the
    same weights whenever only the interface node lies in the strip (N_O = 1)."""
    a = abs(float(xi_h))
    if delta <= 0.0:
        return 1.0 if a < 1.0 else (0.5 if a == 1.0 else 0.0)
    if a <= 1.0 - delta:
        return 1.0
    if a >= 1.0 + delta:
        return 0.0
    if profile == "quintic_halves":
        # a quintic step on each half of the strip, 1/2 on the interface
        if a <= 1.0:
            return 1.0 - 0.5 * quintic((a - 1.0 + delta) / delta)
        return 0.5 * (1.0 - quintic((a - 1.0) / delta))
    if profile == "quintic_normalised":
        # one-sided hat r (1 on the element, 1 - q(d / delta) at distance d outside),
        # divided by the sum over the two subdomains that cover the node
        r = 1.0 - quintic(abs(a - 1.0) / delta)
        return 1.0 / (1.0 + r) if a <= 1.0 else r / (1.0 + r)
    t = (a - 1.0 + delta) / (2.0 * delta)
    if profile == "linear":
        return 1.0 - t
    if profile != "quintic":
        raise ValueError(profile)
    return 1.0 - quintic(t)


def layer_delta(P, n_o, rule="mid"):
    """Overlap half-width (reference units) used for the weights when the
    strip holds N_O node layers.

    Readings (parity unpinned for N_O >= 2; the definition is deferred to an
    earlier paper): rule "mid", the midpoint between the distances of the last
    included (k = N_O - 1) and the first excluded (k = N_O) neighbour node;
    rule "node", the distance of the last included node, so that the weight
    function reaches 0 on the outermost node of the subdomain.  Both are capped
    at 1 (delta_O = dx/2).  Every such choice gives the same weights for
    N_O = 1: face nodes 1/2, the rest of the core 1 (the only case Table 1
    pins, rows 1 vs 3 at P = 4)."""
    xi = gll_nodes(P)
    d = 1.0 + xi
    if n_o <= 0:
        return 0.0
    if n_o >= len(d):
        return 1.0
    if rule == "node":
        return min(d[n_o - 1], 1.0)
    if rule != "mid":
        raise ValueError(rule)
    return min(0.5 * (d[n_o - 1] + d[n_o]), 1.0)


def subdomain_1d(P, n_o, delta, profile="quintic"):
    """One direction of an element-centred subdomain.

    Returns (de, i, w): for each of the m = P + 1 + 2 N_O subdomain nodes, the
    element offset (-1, 0, +1), the node index inside that element and the 1D
    weight.  The left strip is the last N_O nodes of the left neighbour, the
    right strip the first N_O nodes of the right neighbour; xi_H = xi - 2 on the
    left, xi on the core, xi + 2 on the right (Fig. wH).  N_O = 0 gives the
    element alone with weight 1 (block Jacobi)."""
    xi = gll_nodes(P)
    n = P + 1
    de, ii, w = [], [], []
    for i in range(n - n_o, n):
        de.append(-1)
        ii.append(i)
        w.append(hat_weight(xi[i] - 2.0, delta, profile))
    for i in range(n):
        de.append(0)
        ii.append(i)
        w.append(1.0 if n_o == 0 else hat_weight(xi[i], delta, profile))
    for i in range(n_o):
        de.append(1)
        ii.append(i)
        w.append(hat_weight(xi[i] + 2.0, delta, profile))
    return np.array(de), np.array(ii), np.array(w)


def normalised_subdomain_1d(P, n_o, delta, profile="quintic"):
    """subdomain_1d with each weight divided by the sum of the raw weights of
    all subdomains that cover the node (up to three when the strip is wider
    than half an element, as in the "max" overlap of Table 2).  For a strip
    half-width delta <= 1 (reference units) the raw weights of the two
    covering subdomains already sum to one and are returned unchanged.

    Reading (the paper only says the overlap may reach the whole neighbour
    element): a node of an element at reference coordinate xi is seen by the
    subdomain centred o elements away (o = -1, 0, +1) at xi_H = xi - 2 o, and is
    covered by it if it lies in that subdomain's strip."""
    xi = gll_nodes(P)
    n = P + 1
    de, ii, w = subdomain_1d(P, n_o, delta, profile)
    if delta <= 1.0:
        return de, ii, w

    def raw(x):
        return 1.0 if n_o == 0 else hat_weight(x, delta, profile)

    out = np.empty_like(w)
    for a in range(len(de)):
        i = ii[a]
        total = raw(xi[i])                      # own element (o = 0)
        if i >= n - n_o:                        # in the left strip of the subdomain to the right
            total += raw(xi[i] - 2.0)
        if i < n_o:                             # in the right strip of the subdomain to the left
            total += raw(xi[i] + 2.0)
        out[a] = w[a] / total if total > 0 else 0.0
    return de, ii, out


def subdomain_indices(mesh, P, n_o, delta, profile="quintic"):
    """Global indices (Ns x mx my mz, subdomain node (a, b, c) at a + mx (b + my c))
    and the weights W_s = W_z (x) W_y (x) W_x of all subdomains.  n_o and delta
    may be given per direction (tuples of three)."""
    n = P + 1
    B = n ** 3
    n_os = tuple(n_o) if np.ndim(n_o) else (n_o,) * 3
    deltas = tuple(delta) if np.ndim(delta) else (delta,) * 3
    lines = [normalised_subdomain_1d(P, n_os[d], deltas[d], profile) for d in range(3)]
    (dx, ix, wx), (dy, iy, wy), (dz, iz, wz) = lines
    mx, my, mz = len(dx), len(dy), len(dz)
    c, b, a = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
    a, b, c = a.ravel(), b.ravel(), c.ravel()
    ex, ey, ez = mesh.element_coords()
    el = mesh.element(ex[:, None] + dx[a][None, :], ey[:, None] + dy[b][None, :],
                      ez[:, None] + dz[c][None, :])
    local = ix[a] + n * (iy[b] + n * iz[c])
    idx = el * B + local[None, :]
    W = wx[a] * wy[b] * wz[c]
    return idx, W


class LocalSolver:
    """Direct solver of one restricted problem A_ss x = r_s.

    A_ss is badly scaled at high order (the GLL mass weights span two orders
    of magnitude per direction, so its diagonal spans six): the factorisation
    is applied to the symmetrically scaled matrix D A_ss D,
    D = diag(A_ss)^(-1/2), whose condition number is far smaller, and every
    solve ends with iterative refinement steps x += A_ss^{-1} (r - A_ss x)
    (plain FP64 residuals)."""

    def __init__(self, Ass, dense_limit=7000):
        self.m3 = Ass.shape[0]
        self.dscale = 1.0 / np.sqrt(Ass.diagonal())
        Dm = sp.diags(self.dscale)
        Asc = (Dm @ Ass @ Dm).tocsc()
        if self.m3 <= dense_limit:
            self.chol = sla.cho_factor(Asc.toarray(), lower=True)
            self.lu = None
        else:
            self.chol = None
            self.lu = spl.splu(Asc)
        self.Ass = Ass

    def _factor_solve(self, rs):
        b = rs * (self.dscale[:, None] if rs.ndim == 2 else self.dscale)
        y = sla.cho_solve(self.chol, b) if self.chol is not None else self.lu.solve(b)
        return y * (self.dscale[:, None] if rs.ndim == 2 else self.dscale)

    def solve(self, rs, max_refine=40):
        """A_ss^{-1} applied to the columns of rs (m^3 x k): a direct solve
        with the scaled factorisation, then refinement steps until the largest
        relative residual of the columns is below 1e-14 or stops falling by at
        least half (at P = 32 the first solve leaves a residual of about 2e-2
        and 13 steps bring it to 5e-15)."""
        def worst(res):
            return float(np.max(np.linalg.norm(res, axis=0) / np.maximum(np.linalg.norm(rs, axis=0), 1e-300)))

        x = self._factor_solve(rs)
        res = rs - self.Ass @ x
        prev = np.inf
        for _ in range(max_refine):
            rel = worst(res)
            if rel <= 1e-14 or rel > 0.5 * prev:
                break
            prev = rel
            x = x + self._factor_solve(res)
            res = rs - self.Ass @ x
        return x


class SchwarzSmoother:
    """u <- u + sum_s R_s^T W_s A_ss^{-1} R_s (f - A u), repeated nsteps times.

    A_ss = A[I_s, I_s] is extracted from the assembled A.  On the uniform
    periodic mesh it is the same matrix for every s (checked on all subdomains,
    or a sample of ``check`` of them, to 1e-13 relative), so one factorisation
    serves all subdomains.  On a graded mesh (``mesh.graded``) every subdomain
    has its own A_ss and its own factorisation."""

    def __init__(self, A, mesh, P, n_o, delta, profile="quintic", check=64, dense_limit=7000):
        self.idx, self.W = subdomain_indices(mesh, P, n_o, delta, profile)
        self.N = A.shape[0]
        Ns = self.idx.shape[0]
        if getattr(mesh, "graded", False):
            self.solvers = [LocalSolver(A[self.idx[s]][:, self.idx[s]], dense_limit) for s in range(Ns)]
            self.m3 = self.solvers[0].m3
            return
        I0 = self.idx[0]
        Ass = A[I0][:, I0]
        sample = np.arange(Ns) if Ns <= check else np.random.default_rng(0).choice(Ns, check, replace=False)
        ref = abs(Ass).max()
        for s in sample:
            Is = self.idx[s]
            diff = abs(A[Is][:, Is] - Ass).max()
            if diff > 1e-13 * ref:
                raise AssertionError("A_ss differs between subdomains: %g" % diff)
        self.solvers = None
        self.solver = LocalSolver(Ass, dense_limit)
        self.m3 = self.solver.m3
        self.Ass = Ass

    def local_solve(self, rs, max_refine=40):
        """A_ss^{-1} applied to the columns of rs (uniform meshes: the one A_ss)."""
        return self.solver.solve(rs, max_refine)

    def correction(self, r):
        """sum_s R_s^T (W_s A_ss^{-1} R_s r)."""
        rs = r[self.idx]
        if self.solvers is None:
            du = self.local_solve(rs.T).T
        else:
            du = np.stack([self.solvers[s].solve(rs[s][:, None])[:, 0] for s in range(len(self.solvers))])
        return np.bincount(self.idx.ravel(), weights=(du * self.W[None, :]).ravel(), minlength=self.N)

    def smooth(self, A, u, f, nsteps=1):
        for _ in range(nsteps):
            u = u + self.correction(f - A @ u)
        return u


def kron_fdm_correction(mesh, P, n_o, delta, r, factor=2.0, profile="quintic"):
    """sum_s R_s^T W_s A_ss^{-1} R_s r with every A_ss applied by fast
    diagonalisation (Section 3.1): A_ss = Lz (x) My (x) Mx + Mz (x) Ly (x) Mx
    + Mz (x) My (x) Lx over the three 1D lines through the subdomain's
    element, each from the 1D matrices of its direction (``assemble_1d`` or,
    on a graded mesh, ``assemble_1d_graded``) restricted to the subdomain's
    nodes, and inverted with the eigenpairs of L_s S = M_s S Lambda
    (scipy.linalg.eigh).  For large subdomains (m^3 unknowns beyond what a
    direct factorisation handles in seconds); its equality with the direct
    solve of SchwarzSmoother is pinned on small meshes."""
    from .sipg import assemble_1d, assemble_1d_graded

    n = P + 1
    de, ii, _ = subdomain_1d(P, n_o, delta, profile)
    idx, W = subdomain_indices(mesh, P, n_o, delta, profile)
    one_d = []
    for d in range(3):
        if getattr(mesh, "graded", False):
            one_d.append(assemble_1d_graded(mesh.widths[d], P, factor))
        else:
            one_d.append(assemble_1d(mesh.counts[d], mesh.lengths[d], P, factor))
    ex, ey, ez = mesh.element_coords()
    m = len(de)
    cache = {}
    out = np.zeros(len(r))
    for s in range(mesh.num_elements):
        fac = []
        for d, ed in enumerate((ex[s], ey[s], ez[s])):
            key = (d, int(ed))
            if key not in cache:
                L, M = one_d[d]
                g = ((ed + de) % mesh.counts[d]) * n + ii
                lam, S = sla.eigh(L[np.ix_(g, g)], np.diag(M[g]))
                cache[key] = (S, lam)
            fac.append(cache[key])
        (Sx, lx), (Sy, ly), (Sz, lz) = fac
        R = r[idx[s]].reshape(m, m, m)  # (c, b, a)
        V = np.einsum("ap,bq,cr,cba->rqp", Sx, Sy, Sz, R, optimize=True)
        V /= lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
        U = np.einsum("ap,bq,cr,rqp->cba", Sx, Sy, Sz, V, optimize=True).ravel()
        np.add.at(out, idx[s], W * U)
    return out
