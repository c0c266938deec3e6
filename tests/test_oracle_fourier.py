"""Pins for the exact sums f = A fhat and h = A^* f (eq. nfft, eq. nfft*).

Equispaced points turn A into an ordinary DFT matrix (Section 3), so numpy's
FFT is an independent check; single points have closed forms.
"""
import numpy as np

import inputs
from oracle import fourier as FO


def test_index_set_order():
    K = FO.index_set(4, 2)
    assert K.shape == (16, 2)
    assert tuple(K[0]) == (-2, -2) and tuple(K[1]) == (-2, -1) and tuple(K[-1]) == (1, 1)


def test_adjoint_equispaced_is_fft():
    # x_j = j/n, j in I_n: h_k = sum_j f_j exp(-2 pi i k j/n) -- a plain DFT
    n, M = 32, 16
    x = inputs.equispaced(n, 1)
    f = inputs.samples_complex(n, 1)
    j = np.arange(-n // 2, n // 2)
    # reorder f to j = 0..n-1 (index j mod n) and take numpy's FFT
    F = np.fft.fft(np.roll(f, -n // 2))
    k = np.arange(-M // 2, M // 2)
    ref = F[np.mod(k, n)]
    assert np.allclose(FO.adjoint_ndft(x, f, M), ref, atol=1e-11)
    assert np.allclose(j, np.round(x[:, 0] * n))


def test_adjoint_equispaced_2d_is_fft2():
    n, M = 16, 8
    x = inputs.equispaced(n, 2)
    f = inputs.samples_complex(n * n, 3)
    F = np.fft.fft2(np.roll(f.reshape(n, n), (-n // 2, -n // 2), axis=(0, 1)))
    k = np.arange(-M // 2, M // 2)
    ref = F[np.ix_(np.mod(k, n), np.mod(k, n))].ravel()
    assert np.allclose(FO.adjoint_ndft(x, f, M), ref, atol=1e-10)


def test_forward_equispaced_is_ifft():
    n, M = 32, 32
    x = inputs.equispaced(n, 1)
    fh = inputs.coeffs_complex((M,), 5)
    # f_j = sum_k fh_k exp(2 pi i k j / n) = n * ifft of fh placed at k mod n
    a = np.zeros(n, complex)
    a[np.mod(np.arange(-M // 2, M // 2), n)] = fh
    ref = np.roll(n * np.fft.ifft(a), n // 2)
    assert np.allclose(FO.ndft(x, fh, M), ref, atol=1e-11)


def test_single_point_closed_form():
    x = np.array([[0.1234, -0.377]])
    M = 6
    K = FO.index_set(M, 2)
    h = FO.adjoint_ndft(x, np.array([1.0 + 0j]), M)
    assert np.allclose(h, np.exp(-2j * np.pi * (K @ x[0])), atol=1e-14)
    fh = np.zeros(M * M, complex)
    fh[7] = 1.0
    assert np.allclose(FO.ndft(x, fh, M), np.exp(2j * np.pi * (K[7] @ x[0])), atol=1e-14)


def test_adjointness_and_subset():
    x = inputs.random_points(50, 2, 7)
    M = 8
    fh = inputs.coeffs_complex((M * M,), 8)
    f = inputs.samples_complex(50, 9)
    lhs = np.vdot(f, FO.ndft(x, fh, M))            # <A fh, f>
    rhs = np.vdot(FO.adjoint_ndft(x, f, M), fh)    # <fh, A^* f>
    assert abs(lhs - rhs) < 1e-10
    sub = np.array([0, 5, 63, 17])
    assert np.allclose(FO.adjoint_ndft(x, f, M, k_subset=sub), FO.adjoint_ndft(x, f, M)[sub])
    A = FO.matrix_A(x, M)
    assert np.allclose(A @ fh, FO.ndft(x, fh, M))
    assert np.allclose(A.T @ f, FO.transpose_apply(x, f, M))
