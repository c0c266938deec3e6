"""The point-sharded adjoint NFFT through the library's steps (infft_spread_grid,
infft_fft_axis) on one GPU, the ranks emulated in one process: equal to the single-plan
reconstruction to float32 rounding and to the oracle's Algorithm 2.4 (Algorithm 3.7 with
weights)."""
import numpy as np
import pytest

import inputs
from oracle import nfft as NF
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world,M,prec", [(2, 64, "fp32"), (4, 128, "fp32"), (2, 32, "fp64"), (8, 256, "fp32")])
def test_emulated_ranks_match_single_plan(world, M, prec):
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300 import shard as SH
    N = 4 * M * M + 17
    x = inputs.random_points(N, 2, 90 + world)
    f = inputs.samples_complex(N, 91)
    w = inputs.coeffs_complex((N,), 92) / N
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    full = L.Plan(x, M, 2.0, 4, prec)
    full.set_weights(w)
    ref = full.adjoint(to_dev(torch, f, cd), mode=L.MODE_DCF).cpu().numpy()
    ops, fs, plans = [], [], []
    for r in range(world):
        a, b = SH.point_range(N, world, r)
        p = L.Plan(x[a:b], M, 2.0, 4, prec)
        p.set_weights(w[a:b])
        plans.append(p)
        ops.append(SH.GpuOps(p, L.MODE_DCF))
        fs.append(to_dev(torch, f[a:b], cd))
    got = SH.assemble(SH.emulate_ranks(ops, fs, M, full.Ms), M).cpu().numpy()
    tol = 1e-6 if prec == "fp32" else 1e-13
    assert rel(got, ref) < tol
    if M <= 128:
        assert rel(got, NF.adjoint_nfft(x, w * f, M, 2.0, 4).reshape(M, M)) < (1e-5 if prec == "fp32" else 1e-12)


def test_step_calls_reject_bad_arguments():
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300 import api
    x = inputs.random_points(500, 2, 3)
    p = L.Plan(x, 16, 2.0, 4, "fp32")
    t = torch.zeros(32 * 32, dtype=torch.complex64, device="cuda")
    o = torch.zeros(32 * 16, dtype=torch.complex64, device="cuda")
    assert api.infft_fft_axis(p.handle, L.MODE_PLAIN, 32, 1, 3, t.data_ptr(), o.data_ptr(), 0) == L.EINVAL
    assert api.infft_fft_axis(p.handle, L.MODE_DCF, 32, 1, 1, t.data_ptr(), o.data_ptr(), 0) == L.ESTATE
    h = np.zeros(32 * 32, dtype=np.complex64)
    f = torch.zeros(500, dtype=torch.complex64, device="cuda")
    assert api.infft_spread_grid(p.handle, L.MODE_PLAIN, f.data_ptr(), h.ctypes.data, 0) == L.EINVAL


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fft_axis_matches_cufft(prec):
    """infft_fft_axis (the pruned DFT along one axis with the deconvolution of eq. matrix_D)
    against cuFFT (torch.fft) followed by the crop to I_M and the factors 1/(M_sigma w^(k)) of
    the oracle's window transform: the library's FFT cross-checked by another FFT."""
    L, torch = lib_or_skip()
    from oracle import windows as W
    from paper_2302_00414_gb300 import api
    M, m = 64, 4
    p = L.Plan(inputs.random_points(1000, 2, 4), M, 2.0, m, prec)
    Ms = p.Ms
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    k = np.arange(-M // 2, M // 2)
    dinv = 1.0 / (Ms * W.what1(W.KB, k, M, Ms, m))
    g = torch.randn(3, Ms, 5, dtype=cd, device="cuda")
    for nblk in (1, 4):
        out = torch.empty(3 * M * 5, dtype=cd, device="cuda")
        s = api.infft_fft_axis(p.handle, L.MODE_PLAIN, 3, 5, nblk, g.data_ptr(), out.data_ptr(), 0)
        assert s == L.OK, L.last_error()
        ref = torch.fft.fft(g.to(torch.complex128), dim=1).cpu().numpy()[:, np.mod(k, Ms), :] * dinv[None, :, None]
        got = out.cpu().numpy().reshape(nblk, 3, M // nblk, 5).transpose(1, 0, 2, 3).reshape(3, M, 5)
        assert rel(got, ref) < (1e-6 if prec == "fp32" else 1e-13)
