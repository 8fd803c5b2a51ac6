"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each case patches one oracle function with a wrong variant and re-runs a pin
from the other test modules; the pin must raise AssertionError."""
import numpy as np
import pytest

import oracle.schwarz as schwarz
import oracle.sipg as sipg
import test_oracle_max_overlap as tmax
import test_oracle_mg as tmg
import test_oracle_schwarz as tsch
import test_oracle_sipg as tsipg


def _flip_consistency(P, h, d, mu):
    F = _orig_face(P, h, d, mu).tocsr()
    # wrong sign of the consistency/symmetry terms: mu J^T W J + (J^T W G + G^T W J)
    Fmu = _orig_face(P, h, d, 0.0).tocsr()
    return (F - 2 * Fmu).tocoo()


_orig_face = sipg.face_matrix


def test_wrong_face_sign_is_caught(monkeypatch):
    monkeypatch.setattr(sipg, "face_matrix", _flip_consistency)
    with pytest.raises(AssertionError):
        tsipg.test_kronecker_form_eq_A(2)


def test_literal_penalty_formula_is_caught(monkeypatch):
    monkeypatch.setattr(sipg, "stability_threshold", lambda P, h: P * (P + 1) / h)
    with pytest.raises(AssertionError):
        tsipg.test_coercivity_threshold_is_half_of_quoted_formula(4)


def test_interface_weight_one_is_caught(monkeypatch):
    orig = schwarz.hat_weight

    def bad(xi_h, delta, profile="quintic"):
        return 1.0 if abs(abs(xi_h) - 1.0) < 1e-12 else orig(xi_h, delta, profile)
    monkeypatch.setattr(schwarz, "hat_weight", bad)
    with pytest.raises(AssertionError):
        tsch.test_partition_of_unity_node_layers(4, 1, "quintic")


def test_wrong_strip_nodes_are_caught(monkeypatch):
    orig = schwarz.subdomain_1d

    def bad(P, n_o, delta, profile="quintic"):
        de, ii, w = orig(P, n_o, delta, profile)
        ii = np.where(de == 1, P - ii, ii)  # right strip taken from the far side
        return de, ii, w
    monkeypatch.setattr(schwarz, "subdomain_1d", bad)
    with pytest.raises(AssertionError):
        tsch.test_direct_subdomain_inverse_equals_fast_diagonalisation(3, 1)


def test_dropped_volume_direction_is_caught(monkeypatch):
    orig = sipg.volume_matrix

    def bad(P, h):
        K = orig(P, (h[0], h[1], 1e9)).tocsr()  # z-derivative term effectively dropped
        return K.tocoo()
    monkeypatch.setattr(sipg, "volume_matrix", bad)
    with pytest.raises(AssertionError):
        tsipg.test_kronecker_form_eq_A(2)


def _normalise_two_sided_only(P, n_o, delta, profile="quintic"):
    # wrong: the subdomain to the left (whose right strip may also cover the
    # node once the strip is wider than half an element) is left out of the sum
    de, ii, w = schwarz.subdomain_1d(P, n_o, delta, profile)
    if delta <= 1.0:
        return de, ii, w
    xi = schwarz.gll_nodes(P)
    n = P + 1
    out = np.empty_like(w)
    for a in range(len(de)):
        i = ii[a]
        total = schwarz.hat_weight(xi[i], delta, profile)
        if i >= n - n_o:
            total += schwarz.hat_weight(xi[i] - 2.0, delta, profile)
        out[a] = w[a] / total
    return de, ii, out


@pytest.mark.parametrize("bad", [_normalise_two_sided_only,
                                 lambda P, n_o, delta, profile="quintic": schwarz.subdomain_1d(P, n_o, delta, profile)],
                         ids=["two_sided", "unnormalised"])
def test_wrong_max_overlap_normalisation_is_caught(monkeypatch, bad):
    monkeypatch.setattr(schwarz, "normalised_subdomain_1d", bad)
    with pytest.raises(AssertionError):
        tmax.test_partition_of_unity_max_overlap(4, 48, "quintic")


def test_wrong_pcg_beta_sign_is_caught(monkeypatch):
    """The inexact PCG's direction update with a flipped sign of beta (planted
    in the oracle's code) no longer matches textbook PCG."""
    import inspect

    from oracle import multigrid
    from test_oracle_mg import pcg_textbook_gaps
    src = inspect.getsource(multigrid.solve_pcg)
    assert "p = z_new + beta * p" in src
    ns = dict(vars(multigrid))
    exec(compile(src.replace("p = z_new + beta * p", "p = z_new - beta * p"), "<planted>", "exec"), ns)
    monkeypatch.setattr(multigrid, "solve_pcg", ns["solve_pcg"])
    gr, gx, _ = pcg_textbook_gaps(multigrid.solve_pcg)
    assert gr > 1e-3 or gx > 1e-3, (gr, gx)


def test_graded_face_ignoring_the_neighbour_width_is_caught(monkeypatch):
    """A face matrix that gives the e+ side the normal derivative scale of e-
    (one 2/h for both sides) breaks Eq. (A) on a graded mesh."""
    import test_oracle_graded as tgr

    def one_width(P, h, d, mu, h_plus=None):
        return _orig_face(P, h, d, mu)

    monkeypatch.setattr(sipg, "face_matrix", one_width)
    with pytest.raises(AssertionError):
        tgr.test_graded_kronecker_form_eq_A(2)


def test_graded_face_penalty_of_the_mean_width_is_caught(monkeypatch):
    """Taking the penalty of the mean width of the two elements lets a graded
    line become indefinite at the uniform threshold."""
    import test_oracle_graded as tgr

    monkeypatch.setattr(sipg, "face_penalty", lambda P, a, b, factor=2.0: sipg.penalty(P, 0.5 * (a + b), factor))
    with pytest.raises(AssertionError):
        tgr.test_face_penalty_of_the_smaller_width_keeps_the_uniform_threshold(4)
