"""Test helpers: evaluate the oracle on a small periodic patch of elements cut
out of a large mesh, so that full-size GPU results can be checked on sampled
elements.  The operator at an element depends only on it and its six face
neighbours (a 3^3 patch suffices); one Schwarz step at an element depends on
the residual on its 5^3 neighbourhood, i.e. on u and f on a 7^3 patch."""
import numpy as np

from oracle.schwarz import SchwarzSmoother, layer_delta
from oracle.sipg import Mesh, assemble


def element_index(counts, ex, ey, ez):
    nx, ny, nz = counts
    return (ex % nx) + nx * ((ey % ny) + ny * (ez % nz))


def extract_patch(vec, counts, P, e, radius):
    """Values of the (2r+1)^3 elements around element e, in the element order of
    a periodic patch mesh with the same spacing."""
    n3 = (P + 1) ** 3
    nx, ny, nz = counts
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    w = 2 * radius + 1
    out = np.empty(w ** 3 * n3)
    for kz in range(w):
        for ky in range(w):
            for kx in range(w):
                g = element_index(counts, ex + kx - radius, ey + ky - radius, ez + kz - radius)
                p = kx + w * (ky + w * kz)
                out[p * n3:(p + 1) * n3] = vec[g * n3:(g + 1) * n3]
    return out


def patch_mesh(lengths, counts, radius):
    w = 2 * radius + 1
    h = [lengths[d] / counts[d] for d in range(3)]
    return Mesh([w * h[d] for d in range(3)], (w, w, w))


def center(vec, P, radius):
    n3 = (P + 1) ** 3
    w = 2 * radius + 1
    c = radius + w * (radius + w * radius)
    return vec[c * n3:(c + 1) * n3]


def oracle_operator_at(u, lengths, counts, P, e):
    """(A u) restricted to element e, from a 3^3 patch."""
    mesh = patch_mesh(lengths, counts, 1)
    up = extract_patch(u, counts, P, e, 1)
    A = assemble(mesh, P, row_elements=[13])
    return center(A @ up, P, 1)


def oracle_smooth_at(u, f, lengths, counts, P, n_o, e, profile="quintic"):
    """One Schwarz correction sum_s R_s^T W_s A_ss^{-1} R_s (f - A u) at element e, from a 7^3 patch."""
    mesh = patch_mesh(lengths, counts, 3)
    up = extract_patch(u, counts, P, e, 3)
    fp = extract_patch(f, counts, P, e, 3)
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, n_o, layer_delta(P, n_o), profile, check=8)
    return center(sm.correction(fp - A @ up), P, 3)
