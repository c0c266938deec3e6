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


def _real_columns(n_cols=12):
    """Columns of a small random point set with their members' points and l."""
    x, M, sigma, m, Ms = _setup(N=90, M=6, m=2, seed=17)
    members = BO.column_members(x, Ms, m, BO.PATTERN_2M2)
    cols = [c for c in sorted(members) if len(members[c]) >= 2][:n_cols]
    for col in cols:
        js = np.array([j for j, _ in members[col]])
        yield x[js], BO.column_l(col, Ms, 2), M, Ms, m


def real_field_pin_holds() -> bool:
    """Reading R6, real field: b in R^n minimises ||H b - rhs||_2 exactly when the gradient
    of the objective over real b, 2 Re(H^* (H b - rhs)), vanishes (the objective is a convex
    quadratic in b).  Stated from the first-order conditions of the real least-squares
    problem of eqs. 4.10/4.11, not from the oracle's stacked solve; b must also be real."""
    for xm, l, M, Ms, m in _real_columns():
        b, eps = BO.solve_column(xm, l, M, Ms, m, W.KB, field="real")
        H = BO.matrix_H(xm, M)
        r = BO.rhs(l, M, Ms, m, W.KB)
        grad = np.real(np.conj(H).T @ (H @ b - r))
        if np.max(np.abs(b.imag)) != 0.0:
            return False
        if np.max(np.abs(grad)) > 1e-10 * np.linalg.norm(np.conj(H).T @ r):
            return False
        if abs(eps - np.linalg.norm(H @ b - r) ** 2) > 1e-12 * np.linalg.norm(r) ** 2:
            return False
    return True


def test_real_field_first_order_conditions():
    assert real_field_pin_holds()


def test_real_field_single_member_closed_form():
    """One member: min over real b of ||h b - r||^2 is b = Re(h^* r) / ||h||^2, with
    ||h||^2 = |I_M| and h^* r = sum_k w^(k) exp(2 pi i k (x_j - l/Ms)) written out here
    as a direct sum over I_M."""
    M, Ms, m = 8, 16, 3
    xm = np.array([[0.137, -0.402]])
    l = np.array([2, -6])
    b, _ = BO.solve_column(xm, l, M, Ms, m, W.KB, field="real")
    k1 = np.arange(-M // 2, M // 2)
    hr = 0.0 + 0.0j
    for a in k1:
        for c in k1:
            wk = W.what1(W.KB, np.array([a]), M, Ms, m)[0] * W.what1(W.KB, np.array([c]), M, Ms, m)[0]
            hr += wk * np.exp(2j * np.pi * (a * (xm[0, 0] - l[0] / Ms) + c * (xm[0, 1] - l[1] / Ms)))
    assert abs(b[0] - hr.real / M ** 2) < 1e-13 * abs(hr)


def test_real_field_matches_numerical_minimiser():
    """A generic minimiser (BFGS on the real objective, started at 0) reaches the same b."""
    from scipy.optimize import minimize
    for xm, l, M, Ms, m in list(_real_columns(4)):
        b, eps = BO.solve_column(xm, l, M, Ms, m, W.KB, field="real")
        H = BO.matrix_H(xm, M)
        r = BO.rhs(l, M, Ms, m, W.KB)
        obj = lambda v: float(np.linalg.norm(H @ v - r) ** 2)
        jac = lambda v: 2.0 * np.real(np.conj(H).T @ (H @ v - r))
        res = minimize(obj, np.zeros(len(b)), jac=jac, method="BFGS", options={"gtol": 1e-14, "maxiter": 10000})
        assert res.fun >= eps - 1e-10 * np.linalg.norm(r) ** 2
        assert abs(res.fun - eps) <= 1e-8 * np.linalg.norm(r) ** 2


@pytest.mark.parametrize("pattern", [BO.PATTERN_2M2, BO.PATTERN_PAPER])
def test_column_members_of_matches_full_enumeration(pattern):
    x, M, sigma, m, Ms = _setup(N=150, M=6, m=2, seed=5)
    full = BO.column_members(x, Ms, m, pattern)
    assert BO.column_members_of(x, Ms, m, range(Ms * Ms), pattern) == full
    some = [3, 40, 77, 143]
    assert BO.column_members_of(x, Ms, m, some, pattern) == {c: full[c] for c in some if c in full}


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
