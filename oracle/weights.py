"""Density compensation weights for exact reconstruction (Section 3.1).

Corollary 3.4: weights with sum_j w_j exp(2 pi i k x_j) = delta_{0,k} for all
k in I_{2M} (eq. claim_quadrature_coefficients_double) give A^* W A = I and
hence exact reconstruction of trigonometric polynomials of degree M.
Algorithm 3.6 computes them as the minimum-norm solution of the
underdetermined system A_{2M}^T w = e_0 when |I_{2M}| <= N (normal equations
of the second kind, eq. normal_equations_second_kind_double) and as a
least-squares solution when |I_{2M}| > N (normal equations of the first
kind, eq. normal_equations_first_kind_double).  Both are the minimum-norm
least-squares solution of A_{2M}^T w = e_0, which is what ``weights``
returns; ``weights_normal_equations`` follows the two branches of
Algorithm 3.6 with dense Hermitian solves.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .fourier import adjoint_ndft, matrix_A, transpose_apply, index_set


def e0(M2: int, d: int) -> np.ndarray:
    """e_0 = (delta_{0,k})_{k in I_{M2}} in C order."""
    v = np.zeros(M2 ** d, dtype=np.complex128)
    v[int(sum((M2 // 2) * M2 ** (d - 1 - t) for t in range(d)))] = 1.0
    return v


def weights(x: np.ndarray, M: int, rcond: float = 1e-13) -> np.ndarray:
    """Minimum-norm least-squares solution of A_{2M}^T w = e_0 (dense, small sizes)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    At = matrix_A(x, 2 * M).T
    w, *_ = np.linalg.lstsq(At, e0(2 * M, x.shape[1]), rcond=rcond)
    return w


def weights_normal_equations(x: np.ndarray, M: int) -> np.ndarray:
    """Algorithm 3.6 with dense solves.

    |I_2M| <= N: solve A^T conj(A) v = e_0, then w = conj(A) v;
    |I_2M| >  N: solve conj(A) A^T w = conj(A) e_0 = 1_N.
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    N, d = x.shape
    A = matrix_A(x, 2 * M)
    if (2 * M) ** d <= N:
        G = A.T @ np.conj(A)
        v = sla.solve(G, e0(2 * M, d), assume_a="her")
        return np.conj(A) @ v
    G = np.conj(A) @ A.T
    return sla.solve(G, np.ones(N, dtype=np.complex128), assume_a="her")


def residual_vector(x: np.ndarray, w: np.ndarray, M: int) -> np.ndarray:
    """eps_k = sum_j w_j exp(2 pi i k x_j) - delta_{0,k}, k in I_{2M} (eq. residual_lgs)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return transpose_apply(x, w, 2 * M) - e0(2 * M, x.shape[1])


def residual_inf(x: np.ndarray, w: np.ndarray, M: int) -> float:
    """eps = max_{k in I_2M} |eps_k| (used in Theorem 3.14 and Example 5.2)."""
    return float(np.max(np.abs(residual_vector(x, w, M))))


def reconstruct_exact(x: np.ndarray, f: np.ndarray, w: np.ndarray, M: int, k_subset=None) -> np.ndarray:
    """h^w = A^* W f (eq. Fourier_coeffs_nonequi), exact sums."""
    return adjoint_ndft(x, np.asarray(w) * np.asarray(f), M, k_subset=k_subset)


def rel_err(a: np.ndarray, b: np.ndarray, p=2) -> float:
    """e_p = ||a - b||_p / ||b||_p (eq. errors)."""
    a = np.ravel(a)
    b = np.ravel(b)
    return float(np.linalg.norm(a - b, ord=p) / np.linalg.norm(b, ord=p))
