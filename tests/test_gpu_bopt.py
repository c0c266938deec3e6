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
