"""Parity at the size of the batched two-dimensional workload (d=2, M up to 256,
N_i = U(4,6) M_i^2 random points, Kaiser-Bessel m=4, sigma=2, float32 reconstruction):

* one M=256, N=5 M^2 set: all 65,536 coefficients of the density-compensated
  reconstruction (Algorithm 3.7) against the oracle's float64 Algorithm 2.4 applied to
  W f, and 1,024 of them against the exact sums (eq. nfft*);
* the whole 64-set batch replayed as one CUDA graph, as the benchmark times it: every
  coefficient of every set against the oracle's Algorithm 2.4;
* Algorithm 4.3 on one M=256, N=5 M^2 set: 256 random columns against the oracle's
  dense least squares of eq. opt_overdet_columnwise (explicit H_l), and the
  reconstruction of Algorithm 4.4 with those coefficients against the oracle's.

The oracle runs in a spawn pool (started after CUDA, which spawn allows)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import inputs
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu

TOL32 = 1e-5      # float32 spreading against float64, relative l2


def _alg24(args):
    x, c, M = args
    from oracle import nfft as NF
    return NF.adjoint_nfft(x, c, M, 2.0, 4)


def _column(args):
    xm, l, M, Ms, m, b_gpu = args
    from oracle import bopt as BO
    from oracle import windows as W
    b, eps = BO.solve_column(xm, l, M, Ms, m, W.KB)
    eps_gpu = BO.column_residual_of(b_gpu, xm, l, M, Ms, m, W.KB)
    kappa = float(np.linalg.cond(BO.gram_closed_form(xm, M)))
    return eps, eps_gpu, kappa, float(np.linalg.norm(b_gpu - b) / max(np.linalg.norm(b), 1e-300))


def _pool():
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    return mp.get_context("spawn").Pool(min(16, os.cpu_count() or 2))


def _weights(N, seed):
    """Complex weights of the size of density compensation weights (about 1/N)."""
    return inputs.coeffs_complex((N,), seed) * 0.2 / N + 1.0 / N


def test_dcf_full_vector_at_m256():
    L, torch = lib_or_skip()
    from oracle import fourier as FO
    M = 256
    N = 5 * M * M
    x = inputs.random_points(N, 2, 1234)
    w = _weights(N, 1235)
    f = inputs.samples_complex(N, 1236)
    p = L.Plan(x, M, 2.0, 4, "fp32")
    p.set_weights(w)
    h = p.adjoint(to_dev(torch, f.astype(np.complex64)), mode=L.MODE_DCF).cpu().numpy().ravel()
    c = w * f.astype(np.complex64).astype(np.complex128)
    with _pool() as pool:
        ref = pool.map(_alg24, [(x, c, M)])[0]
    assert h.shape == (M * M,)
    assert rel(h, ref) <= TOL32
    ks = np.random.default_rng(5).choice(M * M, size=1024, replace=False)
    exact = FO.adjoint_ndft(x, c, M, k_subset=ks, chunk=16)
    assert rel(h[ks], exact) <= TOL32


def test_batched_graph_all_sets_full_vectors():
    """The benchmark's launch configuration: 64 sets in one graph replay (three branches)."""
    L, torch = lib_or_skip()
    sets = inputs.batch_sets(64, 0)
    plans, fs, hs, cs = [], [], [], []
    for i, (M, x) in enumerate(sets):
        N = x.shape[0]
        w = _weights(N, 5000 + i)
        f = inputs.samples_complex(N, 1000 + i).astype(np.complex64)
        p = L.Plan(x, M, 2.0, 4, "fp32")
        p.set_weights(w)
        plans.append(p)
        fs.append(to_dev(torch, f))
        hs.append(torch.full((M, M), float("nan"), dtype=torch.complex64, device="cuda"))
        cs.append(w * f.astype(np.complex128))
    batch = L.Batch(plans, fs, hs, L.MODE_DCF)
    for _ in range(2):       # a replay must not depend on the previous one
        batch.run()
    torch.cuda.synchronize()
    with _pool() as pool:
        refs = pool.map(_alg24, [(x, c, M) for (M, x), c in zip(sets, cs)])
    errs = [rel(h.cpu().numpy(), r) for h, r in zip(hs, refs)]
    assert max(errs) <= TOL32, max(errs)


def test_bopt_columns_at_m256():
    """Algorithm 4.3 at the batched workload's largest set shape.  Columns hold about 125
    points within 10 x 10 cells; G_l is then numerically singular (cond 1e13 to 1e16), so
    the comparison is on the column objective eps_l of eq. res_opt_columnwise (reading R8):
    the library's b_l, put into the oracle's explicit H_l, must reach the oracle's minimum
    to a small fraction of ||rhs||^2; b itself is compared where cond(G_l) < 1e8."""
    L, torch = lib_or_skip()
    from oracle import bopt as BO
    from oracle import fourier as FO
    from oracle import nfft as NF
    from oracle import windows as W
    M, m = 256, 4
    Ms = 2 * M
    N = 5 * M * M
    x = inputs.random_points(N, 2, 4321)
    p = L.Plan(x, M, 2.0, m, "fp32")
    res_max = p.optimize_B()
    coef = p.get_bopt().reshape(N, 2 * m + 2, 2 * m + 2)
    xw = NF.wrap_points(x)
    cols = np.random.default_rng(7).choice(Ms * Ms, size=256, replace=False)
    mem = BO.column_members_of(xw, Ms, m, cols)
    assert len(mem) >= 250        # random points at 5 per cell leave almost no column empty
    jobs = []
    for col, mm in mem.items():
        js = np.array([j for j, _ in mm])
        b_gpu = np.array([coef[(j,) + s] for j, s in mm])
        jobs.append((xw[js], BO.column_l(col, Ms, 2), M, Ms, m, b_gpu))
    with _pool() as pool:
        out = pool.map(_column, jobs, chunksize=4)
    rhs2 = float(np.sum(W.what(W.KB, FO.index_set(M, 2), M, Ms, m) ** 2))
    eps, eps_gpu, kappa, db = (np.array(v) for v in zip(*out))
    # the library's columns are least-squares solutions to within 1e-6 ||rhs||^2
    assert np.all(eps_gpu <= eps + 1e-6 * rhs2), float(np.max((eps_gpu - eps) / rhs2))
    # and never better than the minimum (the oracle is the definition)
    assert np.all(eps_gpu >= eps - 1e-9 * rhs2)
    good = kappa < 1e8
    if good.any():
        assert np.all(db[good] <= 1e-14 * kappa[good] + 1e-10)
    # the reported maximum covers these columns
    assert res_max >= np.max(eps_gpu) - 1e-6 * rhs2
    # the reconstruction of Algorithm 4.4 with the library's own coefficients (same B_opt
    # on both sides): the BOPT spread at full size
    f = inputs.samples_complex(N, 99).astype(np.complex64)
    h = p.adjoint(to_dev(torch, f), mode=L.MODE_BOPT).cpu().numpy().ravel()
    ref = BO.reconstruct(x, f.astype(np.complex128), coef, M, 2.0, m, W.KB, BO.PATTERN_2M2)
    assert rel(h, ref) <= TOL32
