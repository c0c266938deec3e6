"""NFFT (Algorithm 2.1) and adjoint NFFT (Algorithm 2.4), step by step.

Grids are stored in "I_Msigma order": the entry for l in I_{M_sigma} sits at
position l + M_sigma/2 along every axis (first coordinate slowest).  All
arithmetic is float64 / complex128.

Index sets (eq. indexset_x).  The printed set adds an integer vector z to
M_sigma x_j - l; since l is itself integral that only makes sense as the
periodic shift z in M_sigma Z^d, which is how it is read here: l belongs to
I_{M_sigma,m}(x_j) iff some representative c = l (mod M_sigma) satisfies
|M_sigma x_{j,t} - c_t| <= m for every t.

For the optimisation approach (Section 4) a second, larger sparsity pattern
is available: the 2m+2 consecutive indices c_t = floor(M_sigma x_{j,t}) - m + s,
s = 0..2m+1, per coordinate, which contains the set above.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import windows as W
from .fourier import index_set

PATTERN_PAPER = "paper"
PATTERN_2M2 = "2m+2"


def wrap_points(x: np.ndarray) -> np.ndarray:
    """Representatives of the points in [-1/2, 1/2)^d: x - floor(x + 1/2)."""
    x = np.asarray(x, dtype=np.float64)
    return x - np.floor(x + 0.5)


def slot_count(m: int) -> int:
    """Slots per coordinate used to enumerate candidate indices: 2m+2."""
    return 2 * m + 2


def point_slots(x: np.ndarray, Ms: int, m: int, pattern: str = PATTERN_PAPER):
    """Per point and coordinate, the candidate grid indices and their membership.

    Returns (cand, valid): int arrays of shape (N, d, 2m+2).  cand holds
    c = floor(Ms x) - m + s (not yet reduced mod Ms); valid marks the slots
    that belong to the index set of the chosen pattern.
    """
    xw = wrap_points(x)
    base = np.floor(Ms * xw).astype(np.int64)
    s = np.arange(slot_count(m))
    cand = base[:, :, None] - m + s[None, None, :]
    if pattern == PATTERN_PAPER:
        # |Ms x - c| <= m decided by comparing Ms x with the integers c - m and c + m,
        # so that rounding in a subtraction cannot move a tap across the support edge
        y = (Ms * xw)[:, :, None]
        valid = (y >= cand - m) & (y <= cand + m)
    elif pattern == PATTERN_2M2:
        valid = np.ones(cand.shape, dtype=bool)
    else:
        raise ValueError(pattern)
    return cand, valid


def reduce_index(c: np.ndarray, Ms: int) -> np.ndarray:
    """Representative of c in I_{Ms} = [-Ms/2, Ms/2)."""
    return np.mod(c + Ms // 2, Ms) - Ms // 2


def window_slot_values(kind: str, x: np.ndarray, M: int, Ms: int, m: int, pattern=PATTERN_PAPER):
    """w~_m(x_{j,t} - c/Ms) per point, coordinate and slot, zero outside the index set."""
    xw = wrap_points(x)
    cand, valid = point_slots(xw, Ms, m, pattern)
    vals = W.periodized_truncated(kind, xw[:, :, None] - cand / Ms, M, Ms, m)
    return np.where(valid, vals, 0.0), cand, valid


def spread(x, c, Ms: int, m: int, coeff, cand, valid) -> np.ndarray:
    """g_l = sum_j sum_{slots} coeff[j, s_1..s_d] c_j at l = (cand[j,t,s_t])_t.

    coeff has shape (N, S, ..., S) (d slot axes, S = 2m+2); slots outside the
    index set (valid False) are skipped.  Returns the grid in I_Msigma order.
    """
    N, d = np.asarray(x).shape
    S = slot_count(m)
    g = np.zeros((Ms,) * d, dtype=np.complex128)
    c = np.asarray(c, dtype=np.complex128)
    for slots in itertools.product(range(S), repeat=d):
        ok = np.ones(N, dtype=bool)
        idx = []
        for t, s in enumerate(slots):
            ok &= valid[:, t, s]
            idx.append(reduce_index(cand[:, t, s], Ms) + Ms // 2)
        if not ok.any():
            continue
        val = coeff[(slice(None),) + slots] * c
        np.add.at(g, tuple(i[ok] for i in idx), val[ok])
    return g


def interpolate(g: np.ndarray, x, Ms: int, m: int, coeff, cand, valid) -> np.ndarray:
    """f_j = sum_{slots} coeff[j, s] g_l, l = (cand[j,t,s_t])_t (step 3 of Algorithm 2.1)."""
    N, d = np.asarray(x).shape
    S = slot_count(m)
    out = np.zeros(N, dtype=np.complex128)
    for slots in itertools.product(range(S), repeat=d):
        ok = np.ones(N, dtype=bool)
        idx = []
        for t, s in enumerate(slots):
            ok &= valid[:, t, s]
            idx.append(reduce_index(cand[:, t, s], Ms) + Ms // 2)
        out += np.where(ok, coeff[(slice(None),) + slots] * g[tuple(idx)], 0.0)
    return out


def tensor_coeffs(vals: np.ndarray) -> np.ndarray:
    """Products prod_t vals[j, t, s_t] as an (N, S, ..., S) array."""
    N, d, S = vals.shape
    out = vals[:, 0, :]
    for t in range(1, d):
        out = out[..., None] * vals[:, t, :].reshape((N,) + (1,) * t + (S,))
    return out


def _dft_axis(M: int, Ms: int, sign: int) -> np.ndarray:
    """exp(sign 2 pi i k l / Ms) for k in I_M (rows) and l in I_Ms (columns)."""
    k = np.arange(-M // 2, M // 2)
    l = np.arange(-Ms // 2, Ms // 2)
    return np.exp(sign * 2j * np.pi * np.outer(k, l) / Ms)


def grid_to_coeffs(g: np.ndarray, M: int) -> np.ndarray:
    """sum_{l in I_Ms} g_l exp(-2 pi i k l / Ms) for k in I_M (the d-variate DFT of
    step 2 of Algorithm 2.4, without the factor 1/|I_Ms|), applied axis by axis."""
    Ms = g.shape[0]
    E = _dft_axis(M, Ms, -1)
    out = g
    for t in range(g.ndim):
        out = np.moveaxis(np.tensordot(E, out, axes=([1], [t])), 0, t)
    return out


def coeffs_to_grid(gh: np.ndarray, Ms: int) -> np.ndarray:
    """sum_{k in I_M} gh_k exp(+2 pi i k l / Ms) for l in I_Ms (step 2 of
    Algorithm 2.1 without the factor 1/|I_Ms|), applied axis by axis."""
    M = gh.shape[0]
    E = _dft_axis(M, Ms, +1).T
    out = gh
    for t in range(gh.ndim):
        out = np.moveaxis(np.tensordot(E, out, axes=([1], [t])), 0, t)
    return out


def what_grid(kind: str, M: int, Ms: int, m: int, d: int) -> np.ndarray:
    """w^(k) for k in I_M as a d-dimensional array in C order."""
    return W.what(kind, index_set(M, d), M, Ms, m).reshape((M,) * d)


def adjoint_nfft(x, f, M: int, sigma: float, m: int, kind: str = W.KB) -> np.ndarray:
    """Algorithm 2.4: h~ = D^* F^* B^* f, returned flat in C order over I_M.

    1. g_l = sum_j f_j w~_m(x_j - l/Ms), l in I_Ms (short sums over I_{Ms,m}(x_j));
    2. g^_k = |I_Ms|^{-1} sum_l g_l exp(-2 pi i k l/Ms), k in I_M;
    3. h~_k = g^_k / w^(k).
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d = x.shape[1]
    Ms = W.oversampled_size(M, sigma)
    vals, cand, valid = window_slot_values(kind, x, M, Ms, m)
    g = spread(x, f, Ms, m, tensor_coeffs(vals), cand, valid)
    gh = grid_to_coeffs(g, M) / Ms ** d
    return (gh / what_grid(kind, M, Ms, m, d)).ravel()


def nfft(x, fhat, M: int, sigma: float, m: int, kind: str = W.KB) -> np.ndarray:
    """Algorithm 2.1: f~ = B F D fhat.

    1. g^_k = fhat_k / w^(k) on I_M, zero on I_Ms minus I_M;
    2. g_l = |I_Ms|^{-1} sum_k g^_k exp(2 pi i k l/Ms), l in I_Ms;
    3. f~_j = sum_{l in I_{Ms,m}(x_j)} g_l w~_m(x_j - l/Ms).
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d = x.shape[1]
    Ms = W.oversampled_size(M, sigma)
    gh = np.asarray(fhat, dtype=np.complex128).reshape((M,) * d) / what_grid(kind, M, Ms, m, d)
    g = coeffs_to_grid(gh, Ms) / Ms ** d
    vals, cand, valid = window_slot_values(kind, x, M, Ms, m)
    return interpolate(g, x, Ms, m, tensor_coeffs(vals), cand, valid)


# --- explicit factor matrices (small sizes only) -------------------------------------

def matrix_D(M: int, Ms: int, m: int, d: int, kind: str = W.KB) -> np.ndarray:
    """D = diag(1 / (|I_Ms| w^(k)))_{k in I_M} (eq. matrix_D)."""
    return np.diag(1.0 / (Ms ** d * W.what(kind, index_set(M, d), M, Ms, m)))


def matrix_F(M: int, Ms: int, d: int) -> np.ndarray:
    """F = (exp(2 pi i k l / Ms))_{l in I_Ms, k in I_M} (eq. matrix_F)."""
    L = index_set(Ms, d)
    K = index_set(M, d)
    return np.exp(2j * np.pi * (L @ K.T) / Ms)


def matrix_B(x, M: int, Ms: int, m: int, kind: str = W.KB, pattern=PATTERN_PAPER, coeff=None) -> np.ndarray:
    """B = (w~_m(x_j - l/Ms))_{j, l in I_Ms} (eq. matrix_B), columns in C order over I_Ms.

    With ``coeff`` (shape (N, S, ..., S)) the nonzeros are taken from it instead
    of from the window, on the slots of the given pattern.
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    N, d = x.shape
    vals, cand, valid = window_slot_values(kind, x, M, Ms, m, pattern)
    if coeff is None:
        coeff = tensor_coeffs(vals)
    B = np.zeros((N, Ms ** d), dtype=np.result_type(coeff.dtype, np.float64))
    S = slot_count(m)
    for slots in itertools.product(range(S), repeat=d):
        ok = np.ones(N, dtype=bool)
        col = np.zeros(N, dtype=np.int64)
        for t, s in enumerate(slots):
            ok &= valid[:, t, s]
            col = col * Ms + reduce_index(cand[:, t, s], Ms) + Ms // 2
        rows = np.nonzero(ok)[0]
        B[rows, col[ok]] += coeff[(slice(None),) + slots][ok]
    return B
