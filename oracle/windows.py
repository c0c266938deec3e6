"""Window functions for the NFFT (Section 2.1) and their Fourier transforms.

The paper leaves the window open (Remark 2.2 cites the literature).  Three
windows are provided, all tensor products of a univariate window:

* Kaiser-Bessel, the compactly supported I0 form
      w(x) = I0(beta * sqrt(1 - (M_sigma x / m)^2))  for |M_sigma x| <= m, 0 otherwise,
  with beta = pi m (2 - 1/sigma'), sigma' = M_sigma / M.  Its exact Fourier
  transform is
      w^(k) = (2m/M_sigma) * sinh(sqrt(beta^2 - a^2)) / sqrt(beta^2 - a^2),
      a = 2 pi m k / M_sigma,
  read as sin(sqrt(a^2 - beta^2)) / sqrt(a^2 - beta^2) when a > beta and as
  the limit 1 when a = beta.  Because w has compact support the truncation
  w_m = w (Section 2.1) is exact.
* centred cardinal B-spline of order 2m, w_B(x) = B_{2m}(M_sigma x)
  (eq. window_bspline), with w^_B(k) = (1/M_sigma) sinc(pi k / M_sigma)^{2m}.
* asymmetric Dirichlet kernel w_D = sum_{k in I_M} exp(2 pi i k x)
  (eq. kernel_Dirichlet_asym) with w^_D(k) = 1 on I_M; it is only used through
  w^ (Algorithm 4.3 and the matrix D).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import i0

KB = "kb"
BSPLINE = "bspline"
DIRICHLET = "dirichlet"


def oversampled_size(M: int, sigma: float) -> int:
    """M_sigma = 2 ceil(ceil(sigma M) / 2) (Section 2.1)."""
    return 2 * math.ceil(math.ceil(sigma * M) / 2)


def kb_beta(m: int, M: int, Ms: int) -> float:
    """Kaiser-Bessel shape parameter beta = pi m (2 - M/M_sigma)."""
    return math.pi * m * (2.0 - M / Ms)


def kb_w1(x: np.ndarray, M: int, Ms: int, m: int) -> np.ndarray:
    """Univariate KB window w(x) in torus units, zero outside [-m/Ms, m/Ms]."""
    x = np.asarray(x, dtype=np.float64)
    t = Ms * x / m
    inside = np.abs(t) <= 1.0
    beta = kb_beta(m, M, Ms)
    arg = beta * np.sqrt(np.clip(1.0 - t * t, 0.0, None))
    return np.where(inside, i0(arg), 0.0)


def kb_what1(k: np.ndarray, M: int, Ms: int, m: int) -> np.ndarray:
    """Fourier transform of the univariate KB window at integer frequencies k."""
    k = np.asarray(k, dtype=np.float64)
    beta = kb_beta(m, M, Ms)
    a = 2.0 * np.pi * m * k / Ms
    r = beta * beta - a * a
    out = np.empty_like(a)
    pos = r > 0
    neg = r < 0
    s = np.sqrt(r[pos])
    out[pos] = np.sinh(s) / s
    s = np.sqrt(-r[neg])
    out[neg] = np.sin(s) / s
    out[~(pos | neg)] = 1.0
    return (2.0 * m / Ms) * out


def bspline_centered(y: np.ndarray, order: int) -> np.ndarray:
    """Centred cardinal B-spline B_order(y), support [-order/2, order/2].

    Truncated-power form: B_n(y) = 1/(n-1)! sum_{j=0}^{n} (-1)^j C(n,j) (y + n/2 - j)_+^{n-1}.
    """
    y = np.asarray(y, dtype=np.float64)
    n = order
    acc = np.zeros_like(y)
    for j in range(n + 1):
        z = y + n / 2.0 - j
        acc += (-1) ** j * math.comb(n, j) * np.where(z > 0, z, 0.0) ** (n - 1)
    out = acc / math.factorial(n - 1)
    return np.where(np.abs(y) < n / 2.0, out, 0.0)


def bspline_w1(x: np.ndarray, M: int, Ms: int, m: int) -> np.ndarray:
    """Univariate B-spline window w_B(x) = B_{2m}(M_sigma x) (eq. window_bspline)."""
    return bspline_centered(Ms * np.asarray(x, dtype=np.float64), 2 * m)


def bspline_what1(k: np.ndarray, M: int, Ms: int, m: int) -> np.ndarray:
    """w^_B(k) = (1/M_sigma) sinc(pi k / M_sigma)^{2m}."""
    t = np.pi * np.asarray(k, dtype=np.float64) / Ms
    s = np.where(t == 0.0, 1.0, np.sin(t) / np.where(t == 0.0, 1.0, t))
    return s ** (2 * m) / Ms


def dirichlet_what1(k: np.ndarray, M: int, Ms: int, m: int) -> np.ndarray:
    """w^_D(k) = 1 for k in I_M (Theorem 4.5)."""
    return np.ones_like(np.asarray(k, dtype=np.float64))


def dirichlet_w1(x: np.ndarray, M: int) -> np.ndarray:
    """Univariate asymmetric Dirichlet kernel D_{M/2-1}(x) + exp(-M pi i x)."""
    x = np.asarray(x, dtype=np.float64)
    k = np.arange(-M // 2, M // 2)
    return np.exp(2j * np.pi * np.multiply.outer(x, k)).sum(axis=-1)


_W1 = {KB: kb_w1, BSPLINE: bspline_w1}
_WHAT1 = {KB: kb_what1, BSPLINE: bspline_what1, DIRICHLET: dirichlet_what1}


def w1(kind: str, x, M: int, Ms: int, m: int) -> np.ndarray:
    """Univariate window value w(x) (torus units) of the given kind."""
    return _W1[kind](x, M, Ms, m)


def what1(kind: str, k, M: int, Ms: int, m: int) -> np.ndarray:
    """Univariate Fourier transform w^(k) of the given kind."""
    return _WHAT1[kind](k, M, Ms, m)


def what(kind: str, K: np.ndarray, M: int, Ms: int, m: int) -> np.ndarray:
    """Multivariate w^(k) = prod_t w^(k_t) for the rows k of K."""
    K = np.atleast_2d(K)
    out = np.ones(K.shape[0])
    for t in range(K.shape[1]):
        out = out * what1(kind, K[:, t], M, Ms, m)
    return out


def periodized_truncated(kind: str, y: np.ndarray, M: int, Ms: int, m: int) -> np.ndarray:
    """Univariate w~_m(y) = sum_{r in Z} w_m(y + r) for a window supported in
    [-m/Ms, m/Ms] (Section 2.1).  Requires 2m < Ms so that at most one shift
    contributes; the sum is still taken over r = -2..2."""
    y = np.asarray(y, dtype=np.float64)
    acc = np.zeros_like(y)
    for r in range(-2, 3):
        acc += w1(kind, y + r, M, Ms, m)
    return acc
