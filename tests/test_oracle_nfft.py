"""Pins for the oracle's Algorithms 2.1 and 2.4.

Reference values are the exact sums (eq. nfft, eq. nfft*).  The tolerance is
the Kaiser-Bessel error estimate of the window literature the paper cites
(Remark 2.2): 4 pi (sqrt(m) + m) (1 - 1/sigma)^(1/4) exp(-2 pi m sqrt(1 - 1/sigma)).
"""
import numpy as np
import pytest

import inputs
from oracle import fourier as FO
from oracle import nfft as NF
from oracle import windows as W


def kb_bound(m, sigma):
    s = np.sqrt(1 - 1 / sigma)
    return 4 * np.pi * (np.sqrt(m) + m) * s ** 0.5 * np.exp(-2 * np.pi * m * s)


@pytest.mark.parametrize("d,M,N,sigma,m", [
    (1, 64, 256, 2.0, 4), (1, 64, 256, 2.0, 6), (1, 32, 100, 1.25, 6),
    (2, 16, 600, 2.0, 4), (2, 16, 600, 1.5, 3), (3, 6, 300, 2.0, 2)])
def test_adjoint_nfft_within_window_bound(d, M, N, sigma, m):
    x = inputs.random_points(N, d, 11)
    f = inputs.samples_complex(N, 12)
    ref = FO.adjoint_ndft(x, f, M)
    err = np.linalg.norm(NF.adjoint_nfft(x, f, M, sigma, m) - ref) / np.linalg.norm(ref)
    assert err < kb_bound(m, sigma)


@pytest.mark.parametrize("d,M,N,sigma,m", [(1, 64, 256, 2.0, 6), (2, 16, 500, 2.0, 4), (2, 8, 300, 1.25, 4)])
def test_nfft_within_window_bound(d, M, N, sigma, m):
    x = inputs.random_points(N, d, 21)
    fh = inputs.coeffs_complex((M ** d,), 22)
    ref = FO.ndft(x, fh, M)
    err = np.linalg.norm(NF.nfft(x, fh, M, sigma, m) - ref) / np.linalg.norm(ref)
    assert err < kb_bound(m, sigma)


def test_error_decays_with_m():
    x = inputs.random_points(300, 1, 3)
    f = inputs.samples_complex(300, 4)
    ref = FO.adjoint_ndft(x, f, 32)
    errs = [np.linalg.norm(NF.adjoint_nfft(x, f, 32, 2.0, m) - ref) / np.linalg.norm(ref) for m in (2, 3, 4, 5, 6)]
    assert all(b < a / 10 for a, b in zip(errs, errs[1:]))


def test_single_point_approximation():
    # exp(2 pi i k x) ~ (|I_Ms| w^(k))^{-1} sum_l exp(2 pi i k l/Ms) w~_m(x - l/Ms) (Section 2.1)
    x = np.array([[0.3141, -0.2718]])
    M, sigma, m = 12, 2.0, 6
    K = FO.index_set(M, 2)
    h = NF.adjoint_nfft(x, np.array([1.0 + 0j]), M, sigma, m)
    # pointwise (max-norm) error of one unit sample; the estimate above is stated
    # for the Kaiser-Bessel family, allow a factor 2 for this window's constant
    assert np.max(np.abs(h - np.exp(-2j * np.pi * (K @ x[0])))) < 2 * kb_bound(m, sigma)


def test_factor_matrices_match_algorithms():
    x = inputs.random_points(40, 2, 5)
    M, sigma, m = 6, 2.0, 2
    Ms = W.oversampled_size(M, sigma)
    B = NF.matrix_B(x, M, Ms, m)
    F = NF.matrix_F(M, Ms, 2)
    D = NF.matrix_D(M, Ms, m, 2)
    fh = inputs.coeffs_complex((M * M,), 6)
    f = inputs.samples_complex(40, 7)
    assert np.allclose(B @ F @ D @ fh, NF.nfft(x, fh, M, sigma, m), atol=1e-12)
    assert np.allclose(D.conj().T @ F.conj().T @ B.conj().T @ f, NF.adjoint_nfft(x, f, M, sigma, m), atol=1e-12)
    # rows of B hold at most (2m+1)^d nonzeros (eq. matrix_B)
    assert np.max(np.count_nonzero(B, axis=1)) <= (2 * m + 1) ** 2


def test_wrapping_and_boundary_points():
    # a point just below -1/2 is the torus point just below +1/2 (periodicity)
    M, sigma, m = 16, 2.0, 4
    x1 = np.array([[-0.5 - 1e-3]])
    x2 = np.array([[0.5 - 1e-3]])
    f = np.array([1.0 + 0.5j])
    assert np.allclose(NF.adjoint_nfft(x1, f, M, sigma, m), NF.adjoint_nfft(x2, f, M, sigma, m), atol=1e-12)
    # the origin (duplicates of the polar grid) sits on a grid node: 2m+1 taps per coordinate
    cand, valid = NF.point_slots(np.zeros((1, 2)), 32, 4)
    assert valid[0, 0].sum() == 9
