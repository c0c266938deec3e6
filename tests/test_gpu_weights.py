"""Parity of the CUDA weight solve (Algorithm 3.6) and the density-compensated
reconstruction (Algorithm 3.7) with the FP64 oracle."""
import numpy as np
import pytest

import inputs
from oracle import fourier as FO
from oracle import weights as WT
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu


def kb_bound(m, sigma):
    s = np.sqrt(1 - 1 / sigma)
    return 4 * np.pi * (np.sqrt(m) + m) * s ** 0.5 * np.exp(-2 * np.pi * m * s)


def test_c1_weights_and_exact_reconstruction_fp64():
    """d=1, M=64, N=256 jittered points, sigma=2, m=6, FP64 (the one-dimensional workload)."""
    L, torch = lib_or_skip()
    x = inputs.jittered_1d(256, 0)
    M = 64
    p = L.Plan(x, M, 2.0, 6, "fp64")
    info = p.weights(max_iter=500, rel_tol=1e-14)
    w = p.get_weights()
    w_ref = WT.weights(x, M)
    assert rel(w, w_ref) < 1e-10
    assert info["residual_inf"] < 1e-12
    assert WT.residual_inf(x, w, M) < 1e-12
    fh = inputs.coeffs_complex((M,), 0)
    f = FO.ndft(x, fh, M)
    h = p.adjoint(to_dev(torch, f), mode=L.MODE_DCF).cpu().numpy()
    assert rel(h, fh) < 1e-10          # exact reconstruction (Corollary 3.4), to NFFT accuracy
    assert rel(h, WT.reconstruct_exact(x, f, w, M)) < kb_bound(6, 2.0)


def test_equispaced_weights_one_over_N():
    L, torch = lib_or_skip()
    x = inputs.equispaced(32, 2)
    p = L.Plan(x, 8, 2.0, 4, "fp64")
    p.weights(max_iter=200, rel_tol=1e-14)
    w = p.get_weights()
    assert np.max(np.abs(w - 1.0 / x.shape[0])) < 1e-12


# (d, M, N, m_cg, weight tolerance, residual tolerance): the CG's matrix is exact only to
# the float64 NFFT accuracy of m_cg (about 4e-14 relative at m_cg = 8, 2e-8 at 5, the largest
# a float64 three-dimensional padded tile fits in shared memory); ill-conditioned random sets
# amplify it in the residual
SECOND_KIND = [(2, 8, 600, 8, 1e-8, 1e-9), (2, 16, 1500, 8, 1e-8, 1e-9), (1, 32, 100, 8, 1e-8, 1e-9),
               (3, 4, 700, 5, 1e-5, 1e-6)]


@pytest.mark.parametrize("method", ["nfft", "toeplitz"])
@pytest.mark.parametrize("d,M,N,m_cg,wtol,etol", SECOND_KIND)
def test_second_kind_weights_match_dense_solution(d, M, N, m_cg, wtol, etol, method):
    L, torch = lib_or_skip()
    x = inputs.random_points(N, d, 21)
    p = L.Plan(x, M, 2.0, min(6, M - 1), "fp64")
    info = p.weights(max_iter=2000, rel_tol=1e-13, m_cg=m_cg, method=method)
    w = p.get_weights()
    w_ref = WT.weights(x, M)
    assert rel(w, w_ref) < wtol
    eps = WT.residual_inf(x, w, M)
    assert eps < etol and info["residual_inf"] == pytest.approx(eps, rel=0.5, abs=etol / 100)
    fh = inputs.coeffs_complex((M,) * d, 22)
    f = FO.ndft(x, fh, M)
    # Theorem 3.14(i) on the exact sums with the GPU weights ...
    assert rel(WT.reconstruct_exact(x, f, w, M), fh) <= M ** d * eps + 1e-13
    # ... and the GPU reconstruction adds at most the NFFT approximation error, which scales
    # with sum_j |w_j f_j| (each coefficient's error is at most the window error times it)
    h = p.adjoint(to_dev(torch, f), mode=L.MODE_DCF).cpu().numpy()
    h_exact = WT.reconstruct_exact(x, f, w, M)
    scale = np.sqrt(M ** d) * np.sum(np.abs(w * f))
    assert np.linalg.norm(h.ravel() - h_exact.ravel()) <= kb_bound(min(6, M - 1), 2.0) * scale


@pytest.mark.parametrize("d,M,N,m_cg,wtol,etol", [(2, 32, 6000, 8, 1e-7, 1e-9), (3, 8, 5000, 5, 1e-5, 1e-6)])
def test_toeplitz_and_nfft_products_reach_the_same_weights(d, M, N, m_cg, wtol, etol):
    """Both forms of the CG apply the same matrix A_2M^* A_2M up to NFFT accuracy."""
    L, torch = lib_or_skip()
    x = inputs.random_points(N, d, 23)
    ws, res = [], []
    for method in ("nfft", "toeplitz"):
        p = L.Plan(x, M, 2.0, 4, "fp64")
        info = p.weights(max_iter=3000, rel_tol=1e-13, m_cg=m_cg, method=method)
        ws.append(p.get_weights())
        res.append(info["residual_inf"])
    assert rel(ws[1], ws[0]) < wtol
    assert max(res) < etol


def test_toeplitz_needs_the_second_kind():
    L, torch = lib_or_skip()
    x = inputs.random_points(50, 1, 31)
    p = L.Plan(x, 64, 2.0, 6, "fp64")     # |I_2M| = 128 > N: first kind
    with pytest.raises(L.InfftError):
        p.weights(max_iter=10, method="toeplitz")


def test_first_kind_weights_least_squares():
    L, torch = lib_or_skip()
    x = inputs.random_points(50, 1, 31)
    M = 64  # |I_2M| = 128 > N = 50
    p = L.Plan(x, M, 2.0, 6, "fp64")
    p.weights(max_iter=3000, rel_tol=1e-12)
    w = p.get_weights()
    A = FO.matrix_A(x, 2 * M)
    # normal equations of the first kind: conj(A) A^T w = 1_N
    assert np.max(np.abs(np.conj(A) @ (A.T @ w) - 1.0)) < 1e-7


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_dcf_with_given_weights_matches_exact_sum(prec, tol):
    """Hot-path parity: GPU A^*Wf against the exact sum with the same w."""
    L, torch = lib_or_skip()
    x = inputs.random_points(7000, 2, 41)
    M = 32
    w = inputs.coeffs_complex((7000,), 42) / 7000
    f = inputs.samples_complex(7000, 43)
    p = L.Plan(x, M, 2.0, 6, prec)
    p.set_weights(w)
    assert np.array_equal(p.get_weights(), w)
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    h = p.adjoint(to_dev(torch, f, cd), mode=L.MODE_DCF).cpu().numpy()
    ref = WT.reconstruct_exact(x, f, w, M)
    assert rel(h, ref) < (tol if prec == "fp32" else 1e-9)


def test_capped_cg_returns_its_best_iterate():
    """A capped CG on a badly conditioned grid (polar, Section 5): the weights come from the
    iterate of smallest residual among x_1, x_2, ..., so in the second kind (where the CG
    residual e_0 - A^* A u is -conj(A^T w - e_0)) the 2-norm of A_2M^T w - e_0 never grows as
    max_iter grows, while the last iterate's residual oscillates."""
    L, torch = lib_or_skip()
    x = inputs.polar(128, 64)           # N = 8192 >= |I_2M| = 4096 for M = 32
    p = L.Plan(x, 32, 2.0, 4, "fp32")
    e0 = (np.arange(64 * 64) == (32 * 64 + 32)).astype(float)
    prev = np.inf
    for it in (1, 2, 3, 5, 8, 13, 21, 30):
        info = p.weights(max_iter=it, rel_tol=1e-14)
        assert info["status"] in (L.OK, L.ENOTCONV)
        assert info["iters"] <= it
        w = p.get_weights()
        assert np.all(np.isfinite(w)) and np.any(w != 0)
        r2 = float(np.linalg.norm(FO.transpose_apply(x, w, 64) - e0))
        assert r2 <= prev * (1 + 1e-9) + 1e-12
        assert abs(info["residual_inf"] - np.max(np.abs(FO.transpose_apply(x, w, 64) - e0))) < 1e-6 * max(1, r2)
        prev = r2
