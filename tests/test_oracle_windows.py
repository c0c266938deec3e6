"""Pins for the oracle's window functions (Section 2.1, eq. window_bspline).

The Fourier transforms are checked against numerical quadrature of the
window itself, and the B-spline against scipy's independent B-spline basis.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.interpolate import BSpline

from oracle import windows as W


def _quad_ft(fun, half_width, k):
    """int_{-a}^{a} fun(x) cos(2 pi k x) dx for an even real window."""
    val, _ = integrate.quad(lambda x: fun(x) * np.cos(2 * np.pi * k * x), -half_width, half_width,
                            limit=400, epsabs=0, epsrel=1e-13)
    return val


@pytest.mark.parametrize("M,sigma,m", [(16, 2.0, 4), (32, 1.25, 6), (64, 2.0, 2), (12, 1.0, 4)])
def test_kb_transform_matches_quadrature(M, sigma, m):
    Ms = W.oversampled_size(M, sigma)
    # frequencies on I_M and beyond beta (where the sin form applies)
    ks = np.array([0, 1, M // 4, M // 2 - 1, -M // 2, Ms // 2, Ms])
    closed = W.kb_what1(ks, M, Ms, m)
    for k, c in zip(ks, closed):
        q = _quad_ft(lambda x: float(W.kb_w1(np.array([x]), M, Ms, m)[0]), m / Ms, k)
        assert abs(q - c) <= 1e-10 * abs(W.kb_what1(np.array([0]), M, Ms, m)[0])


def test_kb_transform_positive_on_IM():
    for M, sigma, m in [(64, 2.0, 4), (128, 1.25, 6), (256, 2.0, 6)]:
        Ms = W.oversampled_size(M, sigma)
        k = np.arange(-M // 2, M // 2)
        assert np.all(W.kb_what1(k, M, Ms, m) > 0)


def test_oversampled_size():
    assert W.oversampled_size(64, 2.0) == 128
    assert W.oversampled_size(12, 1.0) == 12
    assert W.oversampled_size(10, 1.25) == 14  # ceil(12.5)=13 -> 14
    assert W.oversampled_size(16, 1.5) == 24


@pytest.mark.parametrize("order", [2, 4, 8])
def test_bspline_matches_scipy(order):
    y = np.linspace(-order / 2 - 0.3, order / 2 + 0.3, 801)
    knots = np.arange(order + 1) - order / 2
    ref = BSpline.basis_element(knots, extrapolate=False)(y)
    ref = np.nan_to_num(ref)
    assert np.max(np.abs(W.bspline_centered(y, order) - ref)) < 1e-12


@pytest.mark.parametrize("M,sigma,m", [(12, 2.0, 2), (16, 1.0, 4)])
def test_bspline_transform_matches_quadrature(M, sigma, m):
    Ms = W.oversampled_size(M, sigma)
    for k in [0, 1, 3, M // 2 - 1]:
        q = _quad_ft(lambda x: float(W.bspline_w1(np.array([x]), M, Ms, m)[0]), m / Ms, k)
        assert abs(q - W.bspline_what1(np.array([k]), M, Ms, m)[0]) < 1e-12


def test_dirichlet_window_values():
    # w_D(x) = D_{M/2-1}(x) + exp(-M pi i x) (eq. kernel_Dirichlet_asym)
    M = 12
    x = np.array([0.013, 0.25, -0.4])
    closed = np.sin((M - 1) * np.pi * x) / np.sin(np.pi * x) + np.exp(-1j * M * np.pi * x)
    assert np.allclose(W.dirichlet_w1(x, M), closed, atol=1e-12)
    assert np.allclose(W.dirichlet_what1(np.arange(-6, 6), M, 24, 2), 1.0)


def test_periodization():
    M, Ms, m = 16, 32, 4
    y = np.array([0.05, 0.05 + 1, 0.05 - 2, 0.5 - 0.01])
    v = W.periodized_truncated(W.KB, y, M, Ms, m)
    assert np.allclose(v[0], v[1]) and np.allclose(v[0], v[2])
    # outside the support (distance > m/Ms from every integer)
    assert v[3] == 0.0
    # closed support: the edge |Ms y| = m is included (I0(0) = 1)
    assert W.periodized_truncated(W.KB, np.array([m / Ms]), M, Ms, m)[0] == pytest.approx(1.0)
