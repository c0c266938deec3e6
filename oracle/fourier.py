"""Exact nonequispaced Fourier sums (Section 2, eq. nfft, eq. nfft*, eq. matrix_A).

All arithmetic in float64 / complex128.  Frequencies k run over
I_M = Z^d cap [-M/2, M/2)^d in C order: the first coordinate is the slowest,
flat index sum_t (k_t + M/2) M^(d-t).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def index_set(M: int, d: int) -> np.ndarray:
    """I_M as an (M^d, d) integer array in C order (Section 2)."""
    if M % 2:
        raise ValueError("M must be even")
    r = np.arange(-M // 2, M // 2)
    mesh = np.meshgrid(*([r] * d), indexing="ij")
    return np.stack([g.ravel() for g in mesh], axis=1)


def matrix_A(x: np.ndarray, M: int) -> np.ndarray:
    """A = (exp(2 pi i k x_j))_{j, k in I_M}, an N x M^d matrix (eq. matrix_A)."""
    K = index_set(M, x.shape[1])
    return np.exp(1j * TWO_PI * (x @ K.T))


def ndft(x: np.ndarray, fhat: np.ndarray, M: int, chunk: int = 4096) -> np.ndarray:
    """f_j = sum_{k in I_M} fhat_k exp(+2 pi i k x_j), j = 1..N (eq. nfft)."""
    x = np.asarray(x, dtype=np.float64)
    K = index_set(M, x.shape[1])
    fhat = np.asarray(fhat, dtype=np.complex128).ravel()
    out = np.empty(x.shape[0], dtype=np.complex128)
    for s in range(0, x.shape[0], chunk):
        out[s:s + chunk] = np.exp(1j * TWO_PI * (x[s:s + chunk] @ K.T)) @ fhat
    return out


def adjoint_ndft(x: np.ndarray, f: np.ndarray, M: int, k_subset=None, chunk: int = 256) -> np.ndarray:
    """h_k = sum_{j=1}^N f_j exp(-2 pi i k x_j), k in I_M (eq. nfft*), i.e. h = A^* f.

    With ``k_subset`` (flat C-order indices into I_M) only those h_k are
    returned, each still the full sum over all N points.
    """
    x = np.asarray(x, dtype=np.float64)
    K = index_set(M, x.shape[1])
    if k_subset is not None:
        K = K[np.asarray(k_subset)]
    f = np.asarray(f, dtype=np.complex128).ravel()
    out = np.empty(K.shape[0], dtype=np.complex128)
    for s in range(0, K.shape[0], chunk):
        out[s:s + chunk] = np.exp(-1j * TWO_PI * (K[s:s + chunk] @ x.T)) @ f
    return out


def transpose_apply(x: np.ndarray, w: np.ndarray, M: int, chunk: int = 256) -> np.ndarray:
    """[A^T w]_k = sum_j w_j exp(+2 pi i k x_j), k in I_M (left side of eq.
    claim_quadrature_coefficients)."""
    x = np.asarray(x, dtype=np.float64)
    K = index_set(M, x.shape[1])
    w = np.asarray(w, dtype=np.complex128).ravel()
    out = np.empty(K.shape[0], dtype=np.complex128)
    for s in range(0, K.shape[0], chunk):
        out[s:s + chunk] = np.exp(1j * TWO_PI * (K[s:s + chunk] @ x.T)) @ w
    return out
