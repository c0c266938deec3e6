"""Optimisation of the sparse matrix B (Section 4, Algorithm 4.3) and the
reconstruction of Algorithm 4.4, from the definitions, and the inverse adjoint NFFT of
Remark 4.6 with the same B_opt.

For every column l in I_{M_sigma} the nonzeros b_l of B_opt solve the least
squares problem (eq. opt_overdet_columnwise)

    minimise || H_l b - |I_Ms|^{-1} D^{-1} f_l ||_2

with H_l = (exp(-2 pi i k x_j))_{k in I_M, j in I_{Ms,m}(l)} (eq. matrix_Hl)
and f_l the l-th column of F^* (eq. matrix_F), so that the right side is
(w^(k) exp(-2 pi i k l / Ms))_{k in I_M}.  Here H_l and the right side are
formed explicitly and the problem is solved by dense least squares; the
closed forms of Remark 4.2 (eq. matrix_normal_equations_overdet and
eq. right_side_normal_equations_overdet) are provided separately so that
tests can check them against the explicit products.

Reading of the coefficient field: the printed minimisation is over real
vectors, the printed solution (eq. solution_overdet) is complex in general.
``complex`` (the printed solution) is the default; ``real`` solves the
real-constrained problem.

Column index sets (eq. indexset_l) are built from the same point-wise
patterns as the NFFT (``nfft.point_slots``): the paper's set, or the 2m+2
slots per coordinate.  B_opt is returned per point and slot, shape
(N, S, ..., S) with S = 2m+2, zero on slots outside the pattern.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import windows as W
from .fourier import index_set
from .nfft import (PATTERN_2M2, PATTERN_PAPER, coeffs_to_grid, grid_to_coeffs, interpolate, point_slots,
                   reduce_index, slot_count, spread, wrap_points, what_grid)


def column_members(x: np.ndarray, Ms: int, m: int, pattern=PATTERN_2M2):
    """I_{Ms,m}(l) for every column: dict flat column index -> list of (j, slot tuple),
    j ascending.  Column index is C order over I_Ms with l_t + Ms/2."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    N, d = x.shape
    cand, valid = point_slots(x, Ms, m, pattern)
    S = slot_count(m)
    cols = {}
    for j in range(N):
        for slots in itertools.product(range(S), repeat=d):
            if not all(valid[j, t, s] for t, s in enumerate(slots)):
                continue
            col = 0
            for t, s in enumerate(slots):
                col = col * Ms + int(reduce_index(cand[j, t, s], Ms)) + Ms // 2
            cols.setdefault(col, []).append((j, slots))
    return cols


def column_members_of(x: np.ndarray, Ms: int, m: int, cols, pattern=PATTERN_2M2):
    """I_{Ms,m}(l) (eq. indexset_l) for the listed flat columns only, in the layout of
    ``column_members``: flat column -> list of (j, slot tuple), j ascending.

    Point j belongs to column l when, along every coordinate, the offset
    (l_t - (floor(Ms x_t) - m)) mod Ms names one of its slots s_t < 2m+2 and that
    slot is in the pattern.  Vectorised over the points, for large point sets."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    N, d = x.shape
    cand, valid = point_slots(x, Ms, m, pattern)
    S = slot_count(m)
    first = cand[:, :, 0]                          # floor(Ms x_t) - m, not reduced
    out = {}
    for col in cols:
        lt = column_l(int(col), Ms, d)
        s = np.mod(lt[None, :] - first, Ms)        # slot of column l along each axis
        ok = np.all(s < S, axis=1)
        js = np.nonzero(ok)[0]
        mem = []
        for j in js:
            slots = tuple(int(v) for v in s[j])
            if all(valid[j, t, st] for t, st in enumerate(slots)):
                mem.append((int(j), slots))
        if mem:
            out[int(col)] = mem
    return out


def column_l(col: int, Ms: int, d: int) -> np.ndarray:
    """The multi-index l in I_Ms of a flat column index."""
    l = []
    for _ in range(d):
        l.append(col % Ms - Ms // 2)
        col //= Ms
    return np.array(l[::-1], dtype=np.int64)


def matrix_H(x_members: np.ndarray, M: int) -> np.ndarray:
    """H_l = (exp(-2 pi i k x_j))_{k in I_M, j} (eq. matrix_Hl)."""
    K = index_set(M, x_members.shape[1])
    return np.exp(-2j * np.pi * (K @ x_members.T))


def rhs(l: np.ndarray, M: int, Ms: int, m: int, kind: str) -> np.ndarray:
    """|I_Ms|^{-1} D^{-1} f_l = (w^(k) exp(-2 pi i k l / Ms))_{k in I_M}."""
    K = index_set(M, len(l))
    return W.what(kind, K, M, Ms, m) * np.exp(-2j * np.pi * (K @ l) / Ms)


def gram_closed_form(x_members: np.ndarray, M: int) -> np.ndarray:
    """H_l^* H_l by eq. matrix_normal_equations_overdet:
    prod_t (D_{M/2-1}(x_h - x_j) + exp(-M pi i (x_h - x_j))), D_{M/2-1}(u) = sin((M-1) pi u)/sin(pi u)
    with the limit M-1 at u in Z."""
    diff = x_members[:, None, :] - x_members[None, :, :]
    s = np.sin(np.pi * diff)
    near = np.abs(s) < 1e-12
    dir_ = np.where(near, (M - 1) * np.cos((M - 1) * np.pi * np.round(diff)) /
                    np.where(near, np.cos(np.pi * np.round(diff)), 1.0),
                    np.sin((M - 1) * np.pi * diff) / np.where(near, 1.0, s))
    return np.prod(dir_ + np.exp(-1j * M * np.pi * diff), axis=2)


def rhs_closed_form(x_members: np.ndarray, l: np.ndarray, M: int, Ms: int, m: int, kind: str) -> np.ndarray:
    """v_l = (sum_{k in I_M} w^(k) exp(2 pi i k (x_j - l/Ms)))_j (eq. right_side_normal_equations_overdet),
    using the tensor structure of w^."""
    k = np.arange(-M // 2, M // 2)
    wh = W.what1(kind, k, M, Ms, m)
    out = np.ones(x_members.shape[0], dtype=np.complex128)
    for t in range(x_members.shape[1]):
        y = x_members[:, t] - l[t] / Ms
        out = out * (np.exp(2j * np.pi * np.outer(y, k)) @ wh)
    return out


def solve_column(x_members: np.ndarray, l: np.ndarray, M: int, Ms: int, m: int, kind: str,
                 field: str = "complex", rcond: float = 1e-12):
    """b_l = argmin ||H_l b - rhs||_2 (minimum norm), and the squared residual eps_l
    (eq. res_opt_columnwise)."""
    H = matrix_H(x_members, M)
    r = rhs(l, M, Ms, m, kind)
    if field == "complex":
        b, *_ = np.linalg.lstsq(H, r, rcond=rcond)
    elif field == "real":
        Hr = np.concatenate([H.real, H.imag], axis=0)
        rr = np.concatenate([r.real, r.imag])
        b, *_ = np.linalg.lstsq(Hr, rr, rcond=rcond)
        b = b.astype(np.complex128)
    else:
        raise ValueError(field)
    eps = float(np.linalg.norm(H @ b - r) ** 2)
    return b, eps


def optimize_B(x: np.ndarray, M: int, sigma: float, m: int, kind: str = W.KB,
               pattern=PATTERN_2M2, field: str = "complex", columns=None):
    """Algorithm 4.3.  Returns (coeff, eps): coeff of shape (N, S, ..., S) holds
    B_opt[j, l] at the slot of column l in point j's pattern; eps maps each
    solved column to its squared residual.  ``columns`` restricts the solve to a
    subset of flat column indices (the other entries stay zero)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    N, d = x.shape
    Ms = W.oversampled_size(M, sigma)
    S = slot_count(m)
    members = column_members(x, Ms, m, pattern)
    coeff = np.zeros((N,) + (S,) * d, dtype=np.complex128)
    eps = {}
    todo = members.keys() if columns is None else [c for c in columns if c in members]
    for col in todo:
        mem = members[col]
        js = np.array([j for j, _ in mem])
        l = column_l(col, Ms, d)
        b, e = solve_column(x[js], l, M, Ms, m, kind, field)
        for (j, slots), bj in zip(mem, b):
            coeff[(j,) + slots] = bj
        eps[col] = e
    return coeff, eps


def reconstruct(x: np.ndarray, f: np.ndarray, coeff: np.ndarray, M: int, sigma: float, m: int,
                kind: str = W.KB, pattern=PATTERN_2M2) -> np.ndarray:
    """Algorithm 4.4: h_opt = D^* F^* B_opt^* f, flat C order over I_M.

    g_l = sum_j conj(B_opt[j, l]) f_j, then the same DFT and division by
    |I_Ms| w^(k) as Algorithm 2.4."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d = x.shape[1]
    Ms = W.oversampled_size(M, sigma)
    cand, valid = point_slots(x, Ms, m, pattern)
    g = spread(x, f, Ms, m, np.conj(coeff), cand, valid)
    gh = grid_to_coeffs(g, M) / Ms ** d
    return (gh / what_grid(kind, M, Ms, m, d)).ravel()


def inverse_adjoint(x: np.ndarray, h: np.ndarray, coeff: np.ndarray, M: int, sigma: float, m: int,
                    kind: str = W.KB, pattern=PATTERN_2M2) -> np.ndarray:
    """Remark 4.6: the inverse adjoint NFFT f = B_opt F D h, an approximate solution of
    A^* f = h (eq. problem_infft*) for |I_M| <= N.

    The same steps as Algorithm 2.1 (division by |I_Ms| w^(k), zero padding, DFT with
    sign +) with the window entries of B replaced by the optimised entries B_opt[j, l]
    (not conjugated)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d = x.shape[1]
    Ms = W.oversampled_size(M, sigma)
    gh = np.asarray(h, dtype=np.complex128).reshape((M,) * d) / what_grid(kind, M, Ms, m, d)
    g = coeffs_to_grid(gh, Ms) / Ms ** d
    cand, valid = point_slots(x, Ms, m, pattern)
    return interpolate(g, x, Ms, m, coeff, cand, valid)


def frobenius_error(x: np.ndarray, M: int, sigma: float, m: int, kind_D: str, B: np.ndarray) -> float:
    """|| A^* B F D - I ||_F (eq. matrixnorms_2d) with explicit matrices."""
    from .fourier import matrix_A
    from .nfft import matrix_D, matrix_F
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d = x.shape[1]
    Ms = W.oversampled_size(M, sigma)
    A = matrix_A(x, M)
    P = np.conj(A).T @ B @ matrix_F(M, Ms, d) @ matrix_D(M, Ms, m, d, kind_D)
    return float(np.linalg.norm(P - np.eye(P.shape[0])))


def column_residual_of(B_col_vals: np.ndarray, x_members: np.ndarray, l: np.ndarray, M: int, Ms: int,
                       m: int, kind: str) -> float:
    """|| H_l b - rhs ||_2^2 for a given column vector b (any feasible column)."""
    H = matrix_H(x_members, M)
    return float(np.linalg.norm(H @ B_col_vals - rhs(l, M, Ms, m, kind)) ** 2)


__all__ = ["column_members", "column_l", "matrix_H", "rhs", "gram_closed_form", "rhs_closed_form",
           "solve_column", "optimize_B", "reconstruct", "inverse_adjoint", "frobenius_error", "column_residual_of",
           "PATTERN_2M2", "PATTERN_PAPER", "wrap_points"]
