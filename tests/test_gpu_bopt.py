"""Parity of the CUDA optimisation of B (Algorithm 4.3) and the reconstruction with
B_opt (Algorithm 4.4) against the FP64 oracle, which forms H_l and the right side
explicitly and solves each column by dense least squares."""
import numpy as np
import pytest

import inputs
from oracle import bopt as BO
from oracle import fourier as FO
from oracle import windows as W
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu

PAT = {"2m+2": 0, "paper": 1}


@pytest.mark.parametrize("d,M,N,m,window,pattern,field", [
    (2, 8, 150, 2, "kb", "2m+2", "complex"),
    (2, 8, 150, 2, "kb", "paper", "complex"),
    (2, 8, 120, 2, "bspline", "paper", "complex"),
    (2, 8, 150, 2, "dirichlet", "2m+2", "complex"),
    (2, 8, 150, 2, "kb", "2m+2", "real"),
])
def test_bopt_coefficients_match_oracle(d, M, N, m, window, pattern, field):
    """Well-conditioned columns (distinct points spread over the window): b itself is unique."""
    L, torch = lib_or_skip()
    x = inputs.random_points(N, d, 5)
    p = L.Plan(x, M, 2.0, m, "fp64", window=window)
    opts = PAT[pattern] | (L.BOPT_REAL if field == "real" else 0)
    res = p.optimize_B(opts)
    c_gpu = p.get_bopt()
    c_ref, eps = BO.optimize_B(x, M, 2.0, m, window, pattern, field)
    assert rel(c_gpu, c_ref) < 1e-8
    scale = np.sum(W.what(window, FO.index_set(M, d), M, 2 * M, m) ** 2)
    assert abs(res - max(eps.values())) < 1e-9 * scale


def test_bopt_ill_conditioned_columns_residual_parity():
    """d=1: ~10 members of a column lie within a quarter period, H_l is a clustered
    Vandermonde matrix and G_l = H_l^* H_l is numerically singular; b is not unique to
    working precision, so the column objective (eq. res_opt_columnwise) and the
    reconstruction are compared instead (reading R8)."""
    L, torch = lib_or_skip()
    d, M, N, m = 1, 16, 40, 3
    x = inputs.random_points(N, d, 5)
    p = L.Plan(x, M, 2.0, m, "fp64")
    res = p.optimize_B()
    c_ref, eps = BO.optimize_B(x, M, 2.0, m, W.KB, BO.PATTERN_2M2)
    scale = np.sum(W.what(W.KB, FO.index_set(M, d), M, 2 * M, m) ** 2)
    assert res <= max(eps.values()) + 1e-6 * scale
    fh = inputs.coeffs_complex((M,), 3)
    f = FO.ndft(x, fh, M)
    h = p.adjoint(to_dev(torch, f), mode=L.MODE_BOPT).cpu().numpy()
    ref = BO.reconstruct(x, f, c_ref, M, 2.0, m, W.KB, BO.PATTERN_2M2)
    assert rel(h, fh) <= rel(ref, fh) + 1e-6


def test_bopt_reconstruction_matches_oracle():
    L, torch = lib_or_skip()
    d, M, N, m = 2, 8, 200, 2
    x = inputs.random_points(N, d, 6)
    fh = inputs.coeffs_complex((M, M), 7)
    f = FO.ndft(x, fh, M)
    # the GPU solves the normal equations by Cholesky, the oracle by lstsq: coefficients
    # agree to about cond(G_l) * 1e-16, here ~1e-11, which bounds the FP64 parity
    for prec, tol in (("fp64", 1e-9), ("fp32", 1e-5)):
        p = L.Plan(x, M, 2.0, m, prec)
        p.optimize_B()
        cd = torch.complex128 if prec == "fp64" else torch.complex64
        h = p.adjoint(to_dev(torch, f, cd), mode=L.MODE_BOPT).cpu().numpy()
        c_ref, _ = BO.optimize_B(x, M, 2.0, m, W.KB, BO.PATTERN_2M2)
        ref = BO.reconstruct(x, f, c_ref, M, 2.0, m, W.KB, BO.PATTERN_2M2)
        assert rel(h, ref) < tol


def test_bopt_improves_on_window_and_bound():
    """Theorem 4.5 on the GPU result: ||h_opt - fhat||^2 <= eps sum_k w^(k)^-2 ||fhat||^2."""
    L, torch = lib_or_skip()
    d, M, N, m = 2, 16, 1500, 3
    x = inputs.random_points(N, d, 8)
    p = L.Plan(x, M, 2.0, m, "fp64")
    eps = p.optimize_B()
    fh = inputs.coeffs_complex((M, M), 9)
    f = FO.ndft(x, fh, M)
    h = p.adjoint(to_dev(torch, f), mode=L.MODE_BOPT).cpu().numpy().ravel()
    wh = W.what(W.KB, FO.index_set(M, 2), M, 2 * M, m)
    assert np.linalg.norm(h - fh.ravel()) ** 2 <= eps * np.sum(wh ** -2.0) * np.linalg.norm(fh) ** 2
    h0 = p.adjoint(to_dev(torch, f)).cpu().numpy().ravel()  # plain adjoint NFFT
    assert np.linalg.norm(h - fh.ravel()) < np.linalg.norm(h0 - fh.ravel())


# --- inverse adjoint NFFT (Remark 4.6) --------------------------------------------------

@pytest.mark.parametrize("window,pattern", [("kb", "2m+2"), ("kb", "paper"), ("dirichlet", "2m+2"),
                                            ("bspline", "paper")])
def test_inverse_adjoint_matches_oracle(window, pattern):
    """f = B_opt F D h on the GPU against the oracle's with its own B_opt (well-conditioned
    columns, so both B_opt agree to about 1e-11)."""
    L, torch = lib_or_skip()
    d, M, N, m = 2, 8, 150, 2
    x = inputs.random_points(N, d, 5)
    h = inputs.coeffs_complex((M, M), 95)
    c_ref, _ = BO.optimize_B(x, M, 2.0, m, window, pattern)
    ref = BO.inverse_adjoint(x, h.ravel(), c_ref, M, 2.0, m, window, pattern)
    for prec, tol in (("fp64", 1e-9), ("fp32", 1e-5)):
        p = L.Plan(x, M, 2.0, m, prec, window=window)
        p.optimize_B(PAT[pattern])
        cd = torch.complex128 if prec == "fp64" else torch.complex64
        f = p.inverse_adjoint(to_dev(torch, h, cd)).cpu().numpy()
        assert rel(f, ref) < tol
        # host buffers give the same result
        f_host = p.inverse_adjoint(h.astype(np.complex128 if prec == "fp64" else np.complex64))
        assert np.array_equal(f_host, f)


def test_inverse_adjoint_solves_the_adjoint_problem():
    """The residual of A^* f = h (eq. problem_infft*) with B_opt is below the window's
    (f = B F D h, the plain NFFT), also in one and three dimensions; the oracle's pins bound
    it by ||A^* B_opt F D - I||_F ||h||."""
    L, torch = lib_or_skip()
    for d, M, N, m in ((1, 16, 64, 3), (2, 8, 200, 2), (3, 4, 300, 1)):
        x = inputs.random_points(N, d, 40 + d)
        h = inputs.coeffs_complex((M,) * d, 96)
        p = L.Plan(x, M, 2.0, m, "fp64")
        p.optimize_B()
        f = p.inverse_adjoint(to_dev(torch, h)).cpu().numpy()
        res = np.linalg.norm(FO.adjoint_ndft(x, f, M) - h.ravel())
        f0 = p.forward(to_dev(torch, h)).cpu().numpy()
        res0 = np.linalg.norm(FO.adjoint_ndft(x, f0, M) - h.ravel())
        assert res < res0


def test_inverse_adjoint_needs_bopt():
    L, torch = lib_or_skip()
    x = inputs.random_points(100, 2, 3)
    p = L.Plan(x, 8, 2.0, 2, "fp64")
    with pytest.raises(L.InfftError):
        p.inverse_adjoint(to_dev(torch, inputs.coeffs_complex((8, 8), 1)))
