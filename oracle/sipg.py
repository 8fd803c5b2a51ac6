"""SIPG discretisation of -lap u = f on a periodic Cartesian box.

Section 2: Poisson problem (Eq. poisson) on the periodic domain
[0,lx] x [0,ly] x [0,lz], a Cartesian mesh of equal cuboids, the tensor-product
GLL nodal basis (Eq. u_h), the interior penalty form (Eq. ip) with GLL
quadrature, giving A u = f (Eq. discrete).  Section 4 fixes the penalty:
mu_* = 2 mu_min,*, mu_min,x = P (P+1) / dx.

Graded meshes (an extension: the paper's grids are uniform, Section 4): the
element widths may vary along each axis, the mesh staying a tensor product
(element (ex, ey, ez) is hx[ex] x hy[ey] x hz[ez]).  The same form and
quadrature apply element by element; the penalty of a face between elements
of widths h- and h+ is the one a uniform mesh of the smaller width would use
(``face_penalty``).

Reading of Eq. (ip): the face integral as printed (+[grad v].{u} + {v}.[grad u])
is not consistent with -lap u = f; this module uses the symmetric interior
penalty form of the reference the paper cites for it (Arnold et al.):

    a(v, u) = sum_e int grad v . grad u
              - int_Gamma ( [v] . {grad u} + {grad v} . [u] )
              + int_Gamma mu [v] . [u],

with {v} = (v- + v+)/2 and [v] = n- v- + n+ v+ as defined in Section 2.  All
faces are interior because the domain is periodic.

The 3D matrix is assembled with element and face loops and 3D (volume) / 2D
(face) GLL quadrature; it is NOT built from the 1D Kronecker factors of Eq. (A),
so that Eq. (A) can be tested against it.  ``assemble_1d`` gives those 1D
factors from the same form in one dimension.

Numbering (element-blocked): element e = ex + nx (ey + ny ez); node (i, j, k)
of element e has global index e (P+1)^3 + i + (P+1) (j + (P+1) k).

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np
import scipy.sparse as sp

from .gll import gll_nodes, gll_weights, diff_matrix


class Mesh:
    """Periodic Cartesian mesh of counts[0] x counts[1] x counts[2] equal
    cuboids on [0, lengths[0]] x [0, lengths[1]] x [0, lengths[2]] (Section 2).

    ``widths``: three sequences of element widths (a graded tensor-product
    mesh); lengths and counts then follow from them and ``h`` is None, so that
    code written for equal cuboids fails on a graded mesh instead of using a
    wrong width.  ``widths`` always holds the per-axis element widths."""

    def __init__(self, lengths=None, counts=None, widths=None):
        if widths is not None:
            self.widths = tuple(np.asarray(w, dtype=np.float64).copy() for w in widths)
            if len(self.widths) != 3 or min(len(w) for w in self.widths) < 1:
                raise ValueError("bad mesh")
            if min(float(w.min()) for w in self.widths) <= 0:
                raise ValueError("bad mesh")
            self.counts = tuple(len(w) for w in self.widths)
            self.lengths = tuple(float(w.sum()) for w in self.widths)
            self.graded = True
            self.h = None
        else:
            self.lengths = tuple(float(v) for v in lengths)
            self.counts = tuple(int(v) for v in counts)
            if min(self.counts) < 1 or min(self.lengths) <= 0:
                raise ValueError("bad mesh")
            self.graded = False
            self.h = tuple(self.lengths[d] / self.counts[d] for d in range(3))
            self.widths = tuple(np.full(self.counts[d], self.h[d]) for d in range(3))
        self.num_elements = self.counts[0] * self.counts[1] * self.counts[2]

    def origins(self, d):
        """Left end of every element along axis d (graded or uniform)."""
        return np.concatenate([[0.0], np.cumsum(self.widths[d])[:-1]])

    def element(self, ex, ey, ez):
        nx, ny, nz = self.counts
        return np.mod(ex, nx) + nx * (np.mod(ey, ny) + ny * np.mod(ez, nz))

    def element_coords(self):
        nx, ny, _ = self.counts
        e = np.arange(self.num_elements)
        return e % nx, (e // nx) % ny, e // (nx * ny)


def stability_threshold(P, h):
    """Coercivity threshold of the face penalty of this form: P (P+1) / (2 h).

    For mu below it the 1D matrix L (and hence A) has a negative eigenvalue,
    above it L is positive semi-definite with the constants as null space (a
    test pins this value)."""
    return P * (P + 1) / (2.0 * h)


def face_penalty(P, h_minus, h_plus, factor=2.0):
    """Penalty of a face between elements of widths h_minus and h_plus along its
    normal: the uniform-mesh penalty of the smaller width.

    Reading (graded meshes are an extension; the paper's penalty is for equal
    elements): the threshold of the form grows like 1/h on each side of the
    face, so the face takes the larger of its two neighbours' values.  It
    reduces to ``penalty`` when the widths are equal."""
    return penalty(P, min(h_minus, h_plus), factor)


def penalty(P, h, factor=2.0):
    """mu = factor * mu_min with mu_min the stability threshold of the form.

    Reading: Section 4 sets mu_* = 2 mu_min,* with mu_min 'the stability
    threshold' and quotes mu_min,x = P (P+1) / dx from an earlier paper.  For the
    form written here ([v] and {.} exactly as defined in Section 2) the
    threshold is P (P+1) / (2 dx): the quoted formula belongs to another
    normalisation of the penalty term.  Taking 'twice the stability threshold'
    as the definition gives mu = P (P+1) / dx; with it the oracle reproduces the
    GLL N_O = 1 rates of Table 1 (rows 1-2) to a few percent, while
    2 P (P+1) / dx gives rates about a third lower."""
    return factor * stability_threshold(P, h)


def local_index(n):
    """Arrays (i, j, k) over the n^3 local nodes in the order i + n (j + n k)."""
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def _node_index(n, d, t, p, s):
    """Local index of the node with index t along axis d and (p, s) along the
    two other axes in increasing axis order."""
    ijk = [None, None, None]
    others = [a for a in range(3) if a != d]
    ijk[d] = t
    ijk[others[0]] = p
    ijk[others[1]] = s
    return ijk[0] + n * (ijk[1] + n * ijk[2])


def volume_matrix(P, h):
    """Element matrix of int grad v . grad u with (P+1)^3-point 3D GLL quadrature.

    The gradient of the basis function phi_I, I = (i, j, k), at the quadrature
    point q = (a, b, c) is tabulated from the nodal property phi_i(x_a) = delta_ia:
    d/dx phi_I(q) = (2/hx) phi_i'(x_a) delta_jb delta_kc, etc.  The matrix is
    sum_d G_d^T W G_d with W the diagonal 3D quadrature weights.
    """
    n = P + 1
    B = n ** 3
    x = gll_nodes(P)
    w = gll_weights(P)
    D = diff_matrix(x)
    qa, qb, qc = local_index(n)
    q_of_axis = (qa, qb, qc)
    wq = (h[0] / 2 * w[qa]) * (h[1] / 2 * w[qb]) * (h[2] / 2 * w[qc])
    W = sp.diags(wq)
    K = sp.csr_matrix((B, B))
    for d in range(3):
        rows, cols, vals = [], [], []
        for t in range(n):
            ijk = [qa, qb, qc]
            ijk = [t * np.ones_like(qa) if a == d else ijk[a] for a in range(3)]
            cols.append(ijk[0] + n * (ijk[1] + n * ijk[2]))
            rows.append(np.arange(B))
            vals.append((2.0 / h[d]) * D[q_of_axis[d], t])
        G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(B, B))
        K = K + G.T @ W @ G
    return K.tocoo()


def face_matrix(P, h, d, mu, h_plus=None):
    """Face terms of the SIPG form on one interface normal to axis d.

    Element e- touches the face with its xi_d = +1 side and e+ with its
    xi_d = -1 side; n- = +e_d, n+ = -e_d.  Columns/rows 0..B-1 are the nodes of
    e-, B..2B-1 those of e+.  With 2D GLL quadrature over the face:
    jump [v] . e_d = v- - v+ and average {dv/dx_d}; the matrix is
    mu J^T W J - J^T W G - G^T W J (rows = test function v, columns = trial u).
    ``h`` are the widths of e-; ``h_plus`` the width of e+ along d (graded
    meshes; default h[d]): each side's normal derivative carries its own 2/h.
    The two elements share the face, so their widths across it are equal.
    """
    n = P + 1
    B = n ** 3
    x = gll_nodes(P)
    w = gll_weights(P)
    D = diff_matrix(x)
    others = [a for a in range(3) if a != d]
    g = 2.0 / h[d]
    gp = g if h_plus is None else 2.0 / h_plus
    Jr, Jc, Jv, Gr, Gc, Gv, wf = [], [], [], [], [], [], []
    q = 0
    for s in range(n):
        for p in range(n):
            wf.append((h[others[0]] / 2 * w[p]) * (h[others[1]] / 2 * w[s]))
            # trace of v- at xi_d = +1 is its node t = P; trace of v+ at xi_d = -1 is node t = 0
            Jr += [q, q]
            Jc += [_node_index(n, d, P, p, s), B + _node_index(n, d, 0, p, s)]
            Jv += [1.0, -1.0]
            for t in range(n):
                Gr += [q, q]
                Gc += [_node_index(n, d, t, p, s), B + _node_index(n, d, t, p, s)]
                Gv += [0.5 * g * D[P, t], 0.5 * gp * D[0, t]]
            q += 1
    Qf = q
    J = sp.csr_matrix((Jv, (Jr, Jc)), shape=(Qf, 2 * B))
    G = sp.csr_matrix((Gv, (Gr, Gc)), shape=(Qf, 2 * B))
    Wf = sp.diags(np.array(wf))
    F = mu * (J.T @ Wf @ J) - J.T @ Wf @ G - G.T @ Wf @ J
    F = F.tocoo()
    F.eliminate_zeros()
    return F


def assemble(mesh, P, factor=2.0, row_elements=None):
    """Global SIPG matrix (CSR, N x N, N = Ne (P+1)^3) by loops over elements
    (volume terms) and over the 3 Ne periodic interfaces (face terms).

    ``row_elements``: if given, only the rows of the nodes of these elements are
    assembled (complete rows, other rows empty); used to evaluate the operator
    on a sample of elements of a large mesh.
    """
    if mesh.graded:
        return _assemble_graded(mesh, P, factor, row_elements)
    n = P + 1
    B = n ** 3
    Ne = mesh.num_elements
    N = Ne * B
    K = volume_matrix(P, mesh.h)
    ex, ey, ez = mesh.element_coords()
    if row_elements is None:
        row_mask = np.ones(Ne, dtype=bool)
    else:
        row_mask = np.zeros(Ne, dtype=bool)
        row_mask[np.asarray(row_elements)] = True
    R, C, V = [], [], []
    vol_el = np.nonzero(row_mask)[0]
    R.append((vol_el[:, None] * B + K.row[None, :]).ravel())
    C.append((vol_el[:, None] * B + K.col[None, :]).ravel())
    V.append(np.broadcast_to(K.data[None, :], (len(vol_el), K.nnz)).ravel())
    for d in range(3):
        F = face_matrix(P, mesh.h, d, penalty(P, mesh.h[d], factor))
        nb = mesh.element(ex + (d == 0), ey + (d == 1), ez + (d == 2))
        minus = np.arange(Ne)
        keep = row_mask[minus] | row_mask[nb]
        minus, plus = minus[keep], nb[keep]
        base_r = np.where(F.row[None, :] < B, minus[:, None] * B, plus[:, None] * B - B)
        base_c = np.where(F.col[None, :] < B, minus[:, None] * B, plus[:, None] * B - B)
        rr = (base_r + F.row[None, :]).ravel()
        cc = (base_c + F.col[None, :]).ravel()
        vv = np.broadcast_to(F.data[None, :], (len(minus), F.nnz)).ravel()
        if row_elements is not None:
            ok = row_mask[rr // B]
            rr, cc, vv = rr[ok], cc[ok], vv[ok]
        R.append(rr)
        C.append(cc)
        V.append(vv)
    A = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(N, N))
    return A.tocsr()


def _assemble_graded(mesh, P, factor, row_elements):
    """``assemble`` on a graded mesh: the same element and face loops, with the
    volume matrix of every element built for its own widths and the face
    matrix of every interface for the widths of its two elements (both
    computed once per distinct set of widths)."""
    n = P + 1
    B = n ** 3
    Ne = mesh.num_elements
    N = Ne * B
    ex, ey, ez = mesh.element_coords()
    coords = (ex, ey, ez)
    hx, hy, hz = mesh.widths
    row_mask = np.ones(Ne, dtype=bool)
    if row_elements is not None:
        row_mask = np.zeros(Ne, dtype=bool)
        row_mask[np.asarray(row_elements)] = True
    vol_cache, face_cache = {}, {}
    R, C, V = [], [], []
    for e in np.nonzero(row_mask)[0]:
        h = (hx[ex[e]], hy[ey[e]], hz[ez[e]])
        if h not in vol_cache:
            vol_cache[h] = volume_matrix(P, h)
        K = vol_cache[h]
        R.append(e * B + K.row)
        C.append(e * B + K.col)
        V.append(K.data)
    for d in range(3):
        nb = mesh.element(ex + (d == 0), ey + (d == 1), ez + (d == 2))
        for e in range(Ne):
            p = nb[e]
            if not (row_mask[e] or row_mask[p]):
                continue
            h = (hx[ex[e]], hy[ey[e]], hz[ez[e]])
            hp = mesh.widths[d][coords[d][p]]
            key = (h, hp, d)
            if key not in face_cache:
                face_cache[key] = face_matrix(P, h, d, face_penalty(P, h[d], hp, factor), h_plus=hp)
            F = face_cache[key]
            rr = np.where(F.row < B, e * B + F.row, p * B + F.row - B)
            cc = np.where(F.col < B, e * B + F.col, p * B + F.col - B)
            vv = F.data
            if row_elements is not None:
                ok = row_mask[rr // B]
                rr, cc, vv = rr[ok], cc[ok], vv[ok]
            R.append(rr)
            C.append(cc)
            V.append(vv)
    A = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(N, N))
    return A.tocsr()


def mass_diagonal(mesh, P):
    """Diagonal of the 3D GLL mass matrix, element-blocked (length Ne (P+1)^3):
    (hx/2 w_i)(hy/2 w_j)(hz/2 w_k) at node (i, j, k) of every element."""
    n = P + 1
    w = gll_weights(P)
    i, j, k = local_index(n)
    if mesh.graded:
        ex, ey, ez = mesh.element_coords()
        hx, hy, hz = (mesh.widths[0][ex], mesh.widths[1][ey], mesh.widths[2][ez])
        return ((hx[:, None] / 2 * w[i][None, :]) * (hy[:, None] / 2 * w[j][None, :])
                * (hz[:, None] / 2 * w[k][None, :])).ravel()
    h = mesh.h
    local = (h[0] / 2 * w[i]) * (h[1] / 2 * w[j]) * (h[2] / 2 * w[k])
    return np.tile(local, mesh.num_elements)


def node_coordinates(mesh, P):
    """Physical coordinates (x, y, z) of all nodes, element-blocked."""
    n = P + 1
    xi = gll_nodes(P)
    i, j, k = local_index(n)
    ex, ey, ez = mesh.element_coords()
    out = []
    for d, (ed, loc) in enumerate(((ex, i), (ey, j), (ez, k))):
        x0 = mesh.origins(d)[ed]
        hd = mesh.widths[d][ed]
        out.append((x0[:, None] + (xi[loc][None, :] + 1.0) * hd[:, None] / 2).ravel())
    return tuple(out)


def weak_rhs(mesh, P, f_nodal):
    """Weak right-hand side b = M f with GLL quadrature (Section 2), made
    compatible with the singular periodic operator.

    Reading (the paper states no rule for the compatibility of f): the
    integral mean of f is removed first (f - (1^T M f)/(1^T M 1)), then the
    rounding-level Euclidean mean of b, so that 1^T b = 0 in floating point.
    """
    m = mass_diagonal(mesh, P)
    f = np.asarray(f_nodal, dtype=np.float64)
    f = f - np.dot(m, f) / np.sum(m)
    b = m * f
    return b - b.mean()


def assemble_1d(n_el, length, P, factor=2.0):
    """1D periodic SIPG stiffness L (dense) and the diagonal of the mass M,
    nodes element-blocked (index e (P+1) + i), from the 1D form of Eq. (ip):
    element blocks (2/h) D^T diag(w) D and, per interface between e and e+1,
    mu J J^T - J G^T - G J^T with J = (e_P; -e_0), G = (g/2)(D[P,:]; D[0,:])."""
    n = P + 1
    h = length / n_el
    g = 2.0 / h
    x = gll_nodes(P)
    w = gll_weights(P)
    D = diff_matrix(x)
    mu = penalty(P, h, factor)
    N = n_el * n
    L = np.zeros((N, N))
    Ke = g * D.T @ np.diag(w) @ D
    for e in range(n_el):
        L[e * n:(e + 1) * n, e * n:(e + 1) * n] += Ke
    for e in range(n_el):
        e2 = (e + 1) % n_el
        idx = np.concatenate([np.arange(e * n, (e + 1) * n), np.arange(e2 * n, (e2 + 1) * n)])
        J = np.zeros(2 * n)
        J[P] = 1.0
        J[n] = -1.0
        G = np.concatenate([0.5 * g * D[P, :], 0.5 * g * D[0, :]])
        F = mu * np.outer(J, J) - np.outer(J, G) - np.outer(G, J)
        L[np.ix_(idx, idx)] += F
    M = np.tile(h / 2 * w, n_el)
    return L, M


def assemble_1d_graded(widths, P, factor=2.0):
    """``assemble_1d`` on a periodic line of elements of the given widths:
    element e contributes (2/h_e) D^T diag(w) D, the interface between e and
    e+1 contributes mu J J^T - J G^T - G J^T with J = (e_P; -e_0),
    G = ((1/h_e) D[P,:]; (1/h_{e+1}) D[0,:]) and mu = face_penalty(h_e, h_{e+1})."""
    widths = np.asarray(widths, dtype=np.float64)
    n_el = len(widths)
    n = P + 1
    x = gll_nodes(P)
    w = gll_weights(P)
    D = diff_matrix(x)
    N = n_el * n
    L = np.zeros((N, N))
    for e in range(n_el):
        g = 2.0 / widths[e]
        L[e * n:(e + 1) * n, e * n:(e + 1) * n] += g * D.T @ np.diag(w) @ D
    for e in range(n_el):
        e2 = (e + 1) % n_el
        idx = np.concatenate([np.arange(e * n, (e + 1) * n), np.arange(e2 * n, (e2 + 1) * n)])
        J = np.zeros(2 * n)
        J[P] = 1.0
        J[n] = -1.0
        G = np.concatenate([D[P, :] / widths[e], D[0, :] / widths[e2]])
        mu = face_penalty(P, widths[e], widths[e2], factor)
        L[np.ix_(idx, idx)] += mu * np.outer(J, J) - np.outer(J, G) - np.outer(G, J)
    M = np.concatenate([widths[e] / 2 * w for e in range(n_el)])
    return L, M
