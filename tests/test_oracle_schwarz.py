"""Pins of the oracle's Schwarz smoother (Section 3.1, Table 1, Fig. wH)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.schwarz import (SchwarzSmoother, hat_weight, layer_delta, layers_from_width, max_layers, quintic,
                            subdomain_1d, subdomain_indices)
from oracle.sipg import Mesh, assemble, assemble_1d
from paper_1612_04796_gb300 import inputs

TABLE1 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_gll.json")))


@pytest.mark.parametrize("row", TABLE1["rows"], ids=lambda r: "row%d" % r["row"])
def test_table1_node_layer_column(row):
    """The N_O column of Table 1 (GLL) follows from the overlap width by counting
    the neighbour nodes within the strip, inclusively, on levels P_l = 2..32."""
    ov = row["overlap"]
    got = []
    for P_l in TABLE1["levels"]:
        if ov == "N_O=1":
            got.append(min(1, max_layers(P_l)))
        else:
            got.append(layers_from_width(P_l, float(ov.split("=")[1])))
    assert got == row["n_o"]


def test_quintic_and_hat_properties():
    t = np.linspace(0, 1, 101)
    np.testing.assert_allclose(quintic(t) + quintic(1 - t), 1.0, atol=1e-15)
    assert quintic(0.0) == 0.0 and quintic(1.0) == 1.0
    for prof in ("quintic", "linear", "quintic_halves", "quintic_normalised"):
        for delta in (0.05, 0.16, 0.5, 1.0):
            assert hat_weight(1.0, delta, prof) == pytest.approx(0.5)
            assert hat_weight(-1.0, delta, prof) == pytest.approx(0.5)
            assert hat_weight(1.0 + delta, delta, prof) == 0.0
            assert hat_weight(1.0 - delta, delta, prof) == 1.0
            for s in np.linspace(0, delta, 7):
                assert hat_weight(1 - s, delta, prof) + hat_weight(1 + s, delta, prof) == pytest.approx(1.0)


@pytest.mark.parametrize("P", [2, 4, 8])
@pytest.mark.parametrize("n_o", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("profile", ["quintic", "linear", "quintic_halves", "quintic_normalised"])
def test_partition_of_unity_node_layers(P, n_o, profile):
    """sum_s R_s^T W_s R_s 1 = 1 (the weighted corrections average, Eq. correction:global)."""
    n_o = min(n_o, max_layers(P))
    mesh = Mesh((1, 1, 1), (3, 4, 3))
    idx, W = subdomain_indices(mesh, P, n_o, layer_delta(P, n_o), profile)
    N = mesh.num_elements * (P + 1) ** 3
    s = np.bincount(idx.ravel(), weights=np.broadcast_to(W, idx.shape).ravel(), minlength=N)
    np.testing.assert_allclose(s, 1.0, atol=1e-14)


@pytest.mark.parametrize("P", [2, 4, 8, 16])
@pytest.mark.parametrize("rel", [0.08, 0.5])
def test_partition_of_unity_geometric(P, rel):
    n_o = min(layers_from_width(P, rel), max_layers(P))
    _, _, w = subdomain_1d(P, n_o, min(2 * rel, 1.0))
    m = len(w)
    n = P + 1
    # 1D: node i of an element receives w[n_o + i] (own), w[n_o + n + i] (left
    # neighbour's right strip) and w[i - (n - n_o)] (right neighbour's left strip)
    tot = np.array([w[n_o + i] + (w[n_o + n + i] if i < n_o else 0.0)
                    + (w[i - (n - n_o)] if i >= n - n_o else 0.0) for i in range(n)])
    np.testing.assert_allclose(tot, 1.0, atol=1e-14)
    # nodes outside the strip carry no weight
    assert m == n + 2 * n_o


def test_n_o_one_weights_pinned():
    """N_O = 1: core 1, both interface nodes 1/2, for any admissible strip width."""
    for P in (2, 4, 8, 16):
        _, _, w = subdomain_1d(P, 1, layer_delta(P, 1))
        expect = np.concatenate([[0.5, 0.5], np.ones(P - 1), [0.5, 0.5]])
        np.testing.assert_allclose(w, expect, atol=1e-15)


@pytest.mark.parametrize("P,n_o", [(2, 1), (3, 1), (4, 2), (4, 1)])
def test_direct_subdomain_inverse_equals_fast_diagonalisation(P, n_o):
    """A_ss^{-1} = (S (x) S (x) S)(I(x)I(x)Lx + I(x)Ly(x)I + Lz(x)I(x)I)^{-1}(S^T (x) S^T (x) S^T)
    with L_s S = M_s S Lambda, S^T M_s S = I from the restricted 1D matrices
    (Section 3.1): pins the oracle's index sets and extraction of A_ss."""
    mesh = Mesh((1.0, 1.5, 0.7), (3, 4, 3))
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, n_o, layer_delta(P, n_o))
    n = P + 1
    SL = []
    for d in range(3):
        L, M = assemble_1d(mesh.counts[d], mesh.lengths[d], P)
        # subdomain around element 1 in 1D: last n_o nodes of element 0, element 1, first n_o of element 2
        idx = np.arange(n - n_o, 2 * n + n_o)
        Ls, Ms = L[np.ix_(idx, idx)], np.diag(M[idx])
        lam, S = sla.eigh(Ls, Ms)
        SL.append((S, lam))
    (Sx, lx), (Sy, ly), (Sz, lz) = SL
    m = len(lx)
    rs = inputs.gaussian(m ** 3, 3)
    R = rs.reshape(m, m, m)  # (c, b, a)
    V = np.einsum("ap,cba->cbp", Sx, R)
    V = np.einsum("bq,cbp->cqp", Sy, V)
    V = np.einsum("cr,cqp->rqp", Sz, V)
    V = V / (lz[:, None, None] + ly[None, :, None] + lx[None, None, :])
    U = np.einsum("cr,rqp->cqp", Sz, V)
    U = np.einsum("bq,cqp->cbp", Sy, U)
    U = np.einsum("ap,cbp->cba", Sx, U)
    direct = sm.local_solve(rs[:, None])[:, 0]
    np.testing.assert_allclose(direct, U.ravel(), rtol=0, atol=1e-11 * np.abs(U).max())


def test_zero_overlap_is_block_jacobi():
    """N_O = 0 with unit weights: the correction is the element-block inverse
    of A applied to the residual (textbook block Jacobi)."""
    mesh = Mesh((1, 1, 1), (3, 3, 3))
    P = 2
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, 0, 0.0)
    B = (P + 1) ** 3
    r = inputs.gaussian(A.shape[0], 5)
    got = sm.correction(r)
    Ad = A.toarray()
    for e in range(mesh.num_elements):
        blk = slice(e * B, (e + 1) * B)
        np.testing.assert_allclose(got[blk], np.linalg.solve(Ad[blk, blk], r[blk]), atol=1e-12)


def test_subdomain_matrices_translation_invariant_and_spd():
    mesh = Mesh((2.0, 1.0, 1.0), (4, 3, 3))
    P = 4
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, 2, layer_delta(P, 2), check=10 ** 6)  # checks every subdomain
    ev = np.linalg.eigvalsh(sm.Ass.toarray())
    assert ev[0] > 0


@pytest.mark.parametrize("P,n_o", [(8, 3), (16, 1)])
def test_local_solve_reaches_rounding_level(P, n_o):
    """The oracle's direct subdomain solve (scaled factorisation plus
    refinement) solves A_ss x = r_s to the FP64 rounding level: residual
    below 1e-14 of the right-hand side on every column, at high order where
    A_ss is badly scaled (Section 3.1, Eq. subproblem)."""
    mesh = Mesh((1.0, 1.5, 0.7), (3, 3, 3))
    A = assemble(mesh, P)
    sm = SchwarzSmoother(A, mesh, P, n_o, layer_delta(P, n_o), check=2)
    rs = inputs.gaussian(sm.m3 * 3, 60).reshape(sm.m3, 3)
    x = sm.local_solve(rs)
    res = np.linalg.norm(rs - sm.Ass @ x, axis=0) / np.linalg.norm(rs, axis=0)
    assert np.all(res < 1e-14), res


def test_layer_delta_readings():
    """The two node-based readings of the weight half-width: "node" is the
    distance of the outermost included neighbour node (its weight becomes 0),
    "mid" lies halfway to the first excluded node; for N_O = 1 both give the
    same weights (face nodes 1/2)."""
    from oracle.gll import gll_nodes
    d = 1.0 + gll_nodes(16)
    assert layer_delta(16, 3, "node") == pytest.approx(d[2])
    assert layer_delta(16, 3, "mid") == pytest.approx(0.5 * (d[2] + d[3]))
    assert hat_weight(1.0 + layer_delta(16, 3, "node"), layer_delta(16, 3, "node")) == 0.0
    for rule in ("node", "mid"):
        de, ii, w = subdomain_1d(8, 1, layer_delta(8, 1, rule))
        np.testing.assert_allclose(w, [0.5] + [0.5] + [1.0] * 7 + [0.5] + [0.5])
