"""Pins for the oracle's matrix optimisation (Section 4, Algorithms 4.3 and 4.4).

* the closed forms of Remark 4.2 equal the explicit products H^* H and H^* rhs;
* each optimised column is no worse than the window's own column (feasible point
  of the same least-squares problem);
* Theorem 4.5 error bound; Example 5.3: ||A^* B_opt F D - I||_F < ||A^* B F D - I||_F.
"""
import numpy as np
import pytest

import inputs
from oracle import bopt as BO
from oracle import fourier as FO
from oracle import nfft as NF
from oracle import windows as W


def _setup(N=120, M=6, sigma=2.0, m=2, seed=81):
    x = NF.wrap_points(inputs.random_points(N, 2, seed))
    return x, M, sigma, m, W.oversampled_size(M, sigma)


def test_closed_forms_match_explicit_products():
    x, M, sigma, m, Ms = _setup()
    members = BO.column_members(x, Ms, m, BO.PATTERN_2M2)
    for col in list(members)[:20]:
        js = np.array([j for j, _ in members[col]])
        l = BO.column_l(col, Ms, 2)
        H = BO.matrix_H(x[js], M)
        assert np.allclose(BO.gram_closed_form(x[js], M), np.conj(H).T @ H, atol=1e-10)
        for kind in (W.KB, W.BSPLINE, W.DIRICHLET):
            v_exp = np.conj(H).T @ BO.rhs(l, M, Ms, m, kind)
            assert np.allclose(BO.rhs_closed_form(x[js], l, M, Ms, m, kind), v_exp, atol=1e-10 * np.abs(v_exp).max())


def test_gram_duplicate_points_limit():
    M = 8
    xm = np.array([[0.1, 0.2], [0.1, 0.2]])
    G = BO.gram_closed_form(xm, M)
    assert np.allclose(G, M * M)  # sum over I_M of 1


@pytest.mark.parametrize("kind", [W.KB, W.BSPLINE])
def test_optimised_columns_beat_window_columns(kind):
    x, M, sigma, m, Ms = _setup()
    coeff, eps = BO.optimize_B(x, M, sigma, m, kind, BO.PATTERN_PAPER)
    vals, cand, valid = NF.window_slot_values(kind, x, M, Ms, m, NF.PATTERN_PAPER)
    orig = NF.tensor_coeffs(vals)
    members = BO.column_members(x, Ms, m, BO.PATTERN_PAPER)
    for col, mem in members.items():
        js = np.array([j for j, _ in mem])
        b0 = np.array([orig[(j,) + s] for j, s in mem])
        l = BO.column_l(col, Ms, 2)
        e0 = BO.column_residual_of(b0, x[js], l, M, Ms, m, kind)
        assert eps[col] <= e0 + 1e-12 * np.sum(np.abs(BO.rhs(l, M, Ms, m, kind)) ** 2)


def test_theorem_4_5_bound_and_reconstruction():
    x, M, sigma, m, Ms = _setup(N=150, M=6, m=2)
    kind = W.KB
    coeff, eps = BO.optimize_B(x, M, sigma, m, kind, BO.PATTERN_2M2)
    fh = inputs.coeffs_complex((M * M,), 82)
    f = FO.ndft(x, fh, M)
    h = BO.reconstruct(x, f, coeff, M, sigma, m, kind, BO.PATTERN_2M2)
    wh = W.what(kind, FO.index_set(M, 2), M, Ms, m)
    bound = max(eps.values()) * np.sum(1.0 / wh ** 2) * np.linalg.norm(fh) ** 2
    assert np.linalg.norm(h - fh) ** 2 <= bound
    # the spread with window coefficients is the plain adjoint NFFT
    vals, cand, valid = NF.window_slot_values(kind, x, M, Ms, m, NF.PATTERN_PAPER)
    h0 = BO.reconstruct(x, f, NF.tensor_coeffs(vals).astype(complex), M, sigma, m, kind, NF.PATTERN_PAPER)
    assert np.allclose(h0, NF.adjoint_nfft(x, f, M, sigma, m, kind), atol=1e-12)


def test_frobenius_matches_columnwise_objective():
    # ||A^* B - |I_Ms|^{-1} D^{-1} F^*||_F^2 = sum_l eps_l (eq. norm_columnwise)
    x, M, sigma, m, Ms = _setup(N=60, M=4, m=2)
    coeff, eps = BO.optimize_B(x, M, sigma, m, W.KB, BO.PATTERN_2M2)
    B = NF.matrix_B(x, M, Ms, m, W.KB, NF.PATTERN_2M2, coeff=coeff)
    A = FO.matrix_A(x, M)
    D = NF.matrix_D(M, Ms, m, 2, W.KB)
    F = NF.matrix_F(M, Ms, 2)
    lhs = np.linalg.norm(np.conj(A).T @ B - np.linalg.inv(D) @ np.conj(F).T / Ms ** 2) ** 2
    # columns without members contribute ||rhs||^2 = sum w^2
    wh2 = np.sum(W.what(W.KB, FO.index_set(M, 2), M, Ms, m) ** 2)
    empty = Ms ** 2 - len(eps)
    assert lhs == pytest.approx(sum(eps.values()) + empty * wh2, rel=1e-8)


@pytest.mark.parametrize("grid", ["mpolar", "jittered"])
def test_example_5_3_optimisation_reduces_frobenius_norm(grid):
    M, sigma, m, R = 12, 2.0, 2, 16
    x = inputs.modified_polar(R, 2 * R) if grid == "mpolar" else inputs.jittered_grid(R, 2, 91)
    x = NF.wrap_points(x)
    Ms = W.oversampled_size(M, sigma)
    B = NF.matrix_B(x, M, Ms, m, W.BSPLINE)
    n = BO.frobenius_error(x, M, sigma, m, W.BSPLINE, B)
    for kind in (W.BSPLINE, W.DIRICHLET):
        coeff, _ = BO.optimize_B(x, M, sigma, m, kind, BO.PATTERN_PAPER)
        Bo = NF.matrix_B(x, M, Ms, m, W.KB, NF.PATTERN_PAPER, coeff=coeff)
        n_opt = BO.frobenius_error(x, M, sigma, m, kind, Bo)
        assert n_opt < n


def test_real_field_variant_is_no_better_than_complex():
    x, M, sigma, m, Ms = _setup(N=80, M=4, m=2)
    _, e_c = BO.optimize_B(x, M, sigma, m, W.KB, BO.PATTERN_2M2, "complex")
    _, e_r = BO.optimize_B(x, M, sigma, m, W.KB, BO.PATTERN_2M2, "real")
    scale = np.sum(W.what(W.KB, FO.index_set(M, 2), M, Ms, m) ** 2)   # ||rhs||^2
    for col in e_c:
        assert e_c[col] <= e_r[col] + 1e-12 * scale


# --- inverse adjoint NFFT (Remark 4.6) --------------------------------------------------

def test_inverse_adjoint_is_the_product_B_F_D():
    """f = B_opt F D h with the explicit factor matrices (eq. matrix_F, eq. matrix_D,
    B_opt placed by eq. matrix_B)."""
    x, M, sigma, m, Ms = _setup(N=80, M=4, m=2)
    for pattern in (BO.PATTERN_2M2, BO.PATTERN_PAPER):
        coeff, _ = BO.optimize_B(x, M, sigma, m, W.KB, pattern)
        h = inputs.coeffs_complex((M * M,), 91)
        f = BO.inverse_adjoint(x, h, coeff, M, sigma, m, W.KB, pattern)
        B = NF.matrix_B(x, M, Ms, m, W.KB, pattern, coeff=coeff)
        f_ref = B @ NF.matrix_F(M, Ms, 2) @ NF.matrix_D(M, Ms, m, 2, W.KB) @ h
        assert np.allclose(f, f_ref, rtol=0, atol=1e-12 * np.abs(f_ref).max())


def test_inverse_adjoint_is_the_adjoint_of_algorithm_4_4():
    """<D^*F^*B^* f, h> = <f, B F D h> for any f, h: the two share B_opt."""
    x, M, sigma, m, Ms = _setup(N=120, M=6, m=2)
    coeff, _ = BO.optimize_B(x, M, sigma, m, W.KB, BO.PATTERN_2M2)
    f = inputs.samples_complex(x.shape[0], 92)
    h = inputs.coeffs_complex((M * M,), 93)
    lhs = np.vdot(BO.reconstruct(x, f, coeff, M, sigma, m, W.KB, BO.PATTERN_2M2), h)
    rhs = np.vdot(f, BO.inverse_adjoint(x, h, coeff, M, sigma, m, W.KB, BO.PATTERN_2M2))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("kind", [W.KB, W.DIRICHLET])
def test_inverse_adjoint_residual_within_frobenius_bound(kind):
    """A^* f - h = (A^* B_opt F D - I) h, so ||A^* f - h|| <= ||A^* B_opt F D - I||_F ||h||
    (eq. problem_infft*, Remark 4.6), and the optimised B does better than the window's."""
    x, M, sigma, m, Ms = _setup(N=200, M=6, m=2)
    coeff, _ = BO.optimize_B(x, M, sigma, m, kind, BO.PATTERN_2M2)
    h = inputs.coeffs_complex((M * M,), 94)
    f = BO.inverse_adjoint(x, h, coeff, M, sigma, m, kind, BO.PATTERN_2M2)
    res = np.linalg.norm(FO.adjoint_ndft(x, f, M) - h)
    # with coeff given, matrix_B takes only the slot positions from the window
    B = NF.matrix_B(x, M, Ms, m, W.KB, BO.PATTERN_2M2, coeff=coeff)
    fro = BO.frobenius_error(x, M, sigma, m, kind, B)
    assert res <= fro * np.linalg.norm(h)
    if kind == W.KB:
        f0 = NF.nfft(x, h, M, sigma, m, kind)          # the window's B, same F and D
        assert res < np.linalg.norm(FO.adjoint_ndft(x, f0, M) - h)
