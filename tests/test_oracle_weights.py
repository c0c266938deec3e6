"""Pins for the oracle's density compensation weights (Section 3.1, Algorithm 3.6).

* equispaced points: F^*F = N I (eq. matrix_product_F*F) makes w_j = 1/N exact;
* Corollary 3.4: A_2M^T w = e_0 gives A^* W A = I and exact reconstruction;
* Example 5.2: exactness for random points while |I_2M| <= N, O(1) errors beyond;
* Theorem 3.14 / 3.15 error and condition bounds in terms of the residual.
"""
import numpy as np
import pytest

import inputs
from oracle import fourier as FO
from oracle import weights as WT


@pytest.mark.parametrize("n,d,M", [(32, 1, 8), (16, 1, 8), (12, 2, 4), (8, 2, 4)])
def test_equispaced_weights_are_one_over_N(n, d, M):
    x = inputs.equispaced(n, d)
    N = n ** d
    assert 2 * M <= n
    for w in (WT.weights(x, M), WT.weights_normal_equations(x, M)):
        assert np.max(np.abs(w - 1.0 / N)) < 1e-14


@pytest.mark.parametrize("d,M,N", [(1, 16, 64), (2, 4, 150), (2, 6, 300)])
def test_corollary_3_4_identity(d, M, N):
    x = inputs.random_points(N, d, 31)
    w = WT.weights(x, M)
    A = FO.matrix_A(x, M)
    assert WT.residual_inf(x, w, M) < 1e-12
    P = np.conj(A).T @ (w[:, None] * A)
    assert np.max(np.abs(P - np.eye(M ** d))) < 1e-12
    # second route through the normal equations of the second kind
    w2 = WT.weights_normal_equations(x, M)
    assert np.max(np.abs(w2 - w)) < 1e-10 * np.max(np.abs(w))


def test_exact_reconstruction_random_trig_poly():
    d, M, N = 2, 6, 260
    x = inputs.random_points(N, d, 41)
    w = WT.weights(x, M)
    for seed in range(3):
        fh = inputs.coeffs_complex((M ** d,), 100 + seed)
        f = FO.ndft(x, fh, M)
        h = WT.reconstruct_exact(x, f, w, M)
        assert WT.rel_err(h, fh) < 1e-12
        assert WT.rel_err(h, fh, np.inf) < 1e-12


def test_example_5_2_threshold_d1():
    # random points, N = 2^(9-d) = 256 for d=1; exact while |I_2M| = 2M < N
    d, N = 1, 256
    x = inputs.random_points(N, d, 51)
    errs = {}
    for M in (16, 64, 256):
        w = WT.weights(x, M)
        fh = inputs.coeffs_real((M,), 52)
        f = FO.ndft(x, fh, M)
        h = WT.reconstruct_exact(x, f, w, M)
        errs[M] = WT.rel_err(h, fh)
        eps = WT.residual_inf(x, w, M)
        # Theorem 3.14(i): e_p <= |I_M| eps
        assert errs[M] <= M * eps * (1 + 1e-6) + 1e-13
        assert WT.rel_err(h, fh, np.inf) <= M * eps * (1 + 1e-6) + 1e-13
    assert errs[16] < 1e-11 and errs[64] < 1e-10
    assert errs[256] > 1e-2


def test_theorem_3_15_condition_bound():
    d, M, N = 1, 8, 40
    x = inputs.random_points(N, d, 61)
    w = WT.weights(x, M)
    r = inputs.rng(62)
    wp = w * (1 + 1e-4 * r.standard_normal(N))     # perturbed weights, nonzero residual
    eps = WT.residual_inf(x, wp, M)
    assert 0 < eps * M < 1
    A = FO.matrix_A(x, M)
    kappa = np.linalg.cond(np.conj(A).T @ (wp[:, None] * A))
    assert 1 <= kappa <= (1 + eps * M) / (1 - eps * M)


def test_first_kind_branch_least_squares():
    # |I_2M| > N: the least-squares solution satisfies the normal equations of the first kind
    d, M, N = 1, 32, 40
    x = inputs.random_points(N, d, 71)
    w = WT.weights(x, M)
    A = FO.matrix_A(x, 2 * M)
    lhs = np.conj(A) @ (A.T @ w)
    assert np.max(np.abs(lhs - np.ones(N))) < 1e-9
    assert np.max(np.abs(WT.weights_normal_equations(x, M) - w)) < 1e-8 * np.max(np.abs(w))
