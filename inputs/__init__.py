"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This module only draws point sets and coefficient vectors.  It holds none of
the inversion method's arithmetic (no window, no Fourier sum, no weights), so
that both the FP64 oracle and the CUDA path can take their inputs from here
without sharing any computation.

Point sets follow the sampling schemes of Section 5 (Remark 5.1) of
Kircheis & Potts, "Fast and direct inversion methods for the multivariate
nonequispaced fast Fourier transform": random, jittered, polar, modified
polar, linogram and golden-angle grids, plus the stack-of-spirals used for
the three-dimensional workload.  Every generator returns a float64 array of
shape (N, d), rows are points, columns are coordinates t = 1..d.  Points are
NOT wrapped into [-1/2, 1/2); the method treats them as points of the torus.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "random_points", "jittered_1d", "jittered_grid", "equispaced",
    "polar", "modified_polar", "linogram", "golden_polar", "spiral_stack",
    "coeffs_complex", "coeffs_real", "samples_complex", "batch_sets",
]


def rng(seed: int) -> np.random.Generator:
    """numpy PCG64 generator for a given integer seed."""
    return np.random.default_rng(int(seed))


def random_points(N: int, d: int, seed: int) -> np.ndarray:
    """Random grid of Remark 5.1(i): x = (eta_1, ..., eta_d) / 2, eta ~ U(-1, 1)."""
    return 0.5 * rng(seed).uniform(-1.0, 1.0, size=(int(N), int(d)))


def jittered_1d(N: int, seed: int, jitter: float = 0.25) -> np.ndarray:
    """One-dimensional jittered points x_j = -1/2 + (j + u_j)/N, u_j ~ U(-jitter, jitter).

    j = 0..N-1.  With u_0 < 0 the first point lies just below -1/2 and is a
    point of the torus near +1/2.
    """
    u = rng(seed).uniform(-jitter, jitter, size=int(N))
    return (-0.5 + (np.arange(N) + u) / N)[:, None]


def jittered_grid(n: int, d: int, seed: int, jitter: float = 0.25) -> np.ndarray:
    """Tensor jittered grid: cell centres of an n^d grid perturbed by U(-jitter, jitter)/n.

    The printed jittered-grid formula of Remark 5.1(i) places points outside the
    torus; this generator keeps its intent (one point per cell of a Cartesian
    grid, randomly displaced inside a neighbourhood of the cell centre).
    """
    r = rng(seed)
    axes = [(-0.5 + (np.arange(n) + 0.5) / n)] * d
    mesh = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([g.ravel() for g in mesh], axis=1)
    return pts + r.uniform(-jitter, jitter, size=pts.shape) / n


def equispaced(n: int, d: int) -> np.ndarray:
    """Equispaced points x = j/n, j in I_n^d (C order, first coordinate slowest)."""
    r = np.arange(-(n // 2), n - n // 2) / n
    mesh = np.meshgrid(*([r] * d), indexing="ij")
    return np.stack([g.ravel() for g in mesh], axis=1)


def polar(n_angles: int, n_radii: int) -> np.ndarray:
    """Polar grid (eq. polar_grid): signed radius r_j = j/n_radii, j in I_{n_radii},
    angle theta_t = pi t / n_angles, t in I_{n_angles}; x = r (cos theta, sin theta).

    Points are ordered angle-major.  N = n_angles * n_radii.
    """
    t = np.arange(-(n_angles // 2), n_angles - n_angles // 2)
    j = np.arange(-(n_radii // 2), n_radii - n_radii // 2)
    theta = np.pi * t / n_angles
    r = j / n_radii
    th, rr = np.meshgrid(theta, r, indexing="ij")
    return np.stack([(rr * np.cos(th)).ravel(), (rr * np.sin(th)).ravel()], axis=1)


def modified_polar(R: int, T: int) -> np.ndarray:
    """Modified polar grid (eq. mpolar_grid): radii j/R for j in I_{floor(sqrt(2) R)}
    (rounded to even), angles pi t/T, t in I_T, keeping only points in [-1/2, 1/2)^2."""
    Rm = int(np.floor(np.sqrt(2.0) * R))
    Rm += Rm % 2
    t = np.arange(-(T // 2), T - T // 2)
    j = np.arange(-(Rm // 2), Rm - Rm // 2)
    th, rr = np.meshgrid(np.pi * t / T, j / R, indexing="ij")
    pts = np.stack([(rr * np.cos(th)).ravel(), (rr * np.sin(th)).ravel()], axis=1)
    keep = np.all((pts >= -0.5) & (pts < 0.5), axis=1)
    return pts[keep]


def linogram(R: int, T: int) -> np.ndarray:
    """Linogram (pseudo-polar) grid (eq. linogram_grid): the two point families
    (j/R, 4t/T * j/R) and (-4t/T * j/R, j/R) for j in I_R, t in I_{T/2}.  N = R*T."""
    j = np.arange(-(R // 2), R - R // 2) / R
    t = np.arange(-(T // 4), T // 2 - T // 4) * 4.0 / T
    jj, tt = np.meshgrid(j, t, indexing="ij")
    bh = np.stack([jj.ravel(), (tt * jj).ravel()], axis=1)
    bv = np.stack([(-tt * jj).ravel(), jj.ravel()], axis=1)
    return np.concatenate([bh, bv], axis=0)


def golden_polar(R: int, T: int) -> np.ndarray:
    """Golden-angle polar grid (eq. golden_angles): polar radii j/R, j in I_R, with
    angles theta_t = mod(pi/2 + t * 2 pi/(1+sqrt 5), pi) - pi/2, t = 0..T-1."""
    t = np.arange(T)
    theta = np.mod(np.pi / 2 + t * 2 * np.pi / (1 + np.sqrt(5.0)), np.pi) - np.pi / 2
    r = np.arange(-(R // 2), R - R // 2) / R
    th, rr = np.meshgrid(theta, r, indexing="ij")
    return np.stack([(rr * np.cos(th)).ravel(), (rr * np.sin(th)).ravel()], axis=1)


def spiral_stack(planes: int = 64, per_plane: int = 32768, turns: int = 64) -> np.ndarray:
    """Stack of Archimedean spirals: planes z_p = -1/2 + p/planes, p = 0..planes-1;
    on each plane s = 0..per_plane-1, r = s/(2 per_plane) in [0, 1/2),
    phi = 2 pi turns s/per_plane.  Columns are (z, y, x)."""
    s = np.arange(per_plane)
    r = s / (2.0 * per_plane)
    phi = 2.0 * np.pi * turns * s / per_plane
    y = r * np.sin(phi)
    x = r * np.cos(phi)
    z = -0.5 + np.arange(planes) / planes
    zz = np.repeat(z, per_plane)
    return np.stack([zz, np.tile(y, planes), np.tile(x, planes)], axis=1)


def coeffs_complex(shape, seed: int) -> np.ndarray:
    """Complex coefficients with Re, Im ~ U(-1, 1) (complex128)."""
    r = rng(seed)
    return r.uniform(-1, 1, size=shape) + 1j * r.uniform(-1, 1, size=shape)


def coeffs_real(shape, seed: int, lo: float = 1.0, hi: float = 10.0) -> np.ndarray:
    """Real coefficients ~ U(lo, hi) as complex128 (Example 5.2 uses U[1, 10])."""
    return rng(seed).uniform(lo, hi, size=shape).astype(np.complex128)


def samples_complex(N: int, seed: int) -> np.ndarray:
    """Measurement vector f with Re, Im ~ U(-1, 1) (complex128)."""
    return coeffs_complex((int(N),), seed)


def batch_sets(count: int, seed: int, Ms=(32, 64, 128, 256), lo: float = 4.0, hi: float = 6.0):
    """Batched two-dimensional workload: `count` independent random point sets.

    For set i the degree M_i is drawn uniformly from `Ms` and the point count
    N_i = floor(U(lo, hi) * M_i^2); points are i.i.d. U[-1/2, 1/2)^2.  Set i uses
    seed (seed * 1000 + i).  Returns a list of (M_i, x_i) pairs.
    """
    r = rng(seed)
    out = []
    for i in range(count):
        M = int(r.choice(Ms))
        N = int(np.floor(r.uniform(lo, hi) * M * M))
        out.append((M, random_points(N, 2, seed * 1000 + i)))
    return out
