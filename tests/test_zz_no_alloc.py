"""The allocation-free reconstruction entry point, infft_adjoint_noalloc.

Some callers cannot allocate device memory during a call (an external allocator
owns the device memory, or cudaMalloc's synchronisation is not acceptable in their
loop).  infft_adjoint_noalloc serves them from a fixed scratch array inside the
library.  This file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.  It also passes in a
fresh process on its own.

Every case runs two calls in a row (the array keeps the previous call's contents) and
compares each with infft_adjoint on the same plan and with the oracle's float64
Algorithm 2.4 (Algorithm 4.4 for B_opt).  The cases cover each scratch layout: d=1 (no
FFT intermediates), d=2, d=3 (both intermediates) and B_opt's padded tiles of edge
T + 2m + 1.
"""
import numpy as np
import pytest

import inputs
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    # d, M, N, m, precision, mode
    (2, 64, 20000, 4, "fp32", "dcf"),
    (2, 64, 20000, 4, "fp64", "plain"),
    (1, 64, 700, 6, "fp64", "dcf"),
    (1, 128, 3000, 4, "fp32", "plain"),
    (3, 16, 12000, 4, "fp32", "dcf"),
    (3, 16, 6000, 3, "fp64", "plain"),
    (2, 16, 1500, 3, "fp64", "bopt"),
    (2, 16, 1500, 3, "fp32", "bopt"),
]


@pytest.mark.parametrize("d,M,N,m,prec,mode", CASES)
def test_noalloc_matches_adjoint_and_oracle_two_calls(d, M, N, m, prec, mode):
    L, torch = lib_or_skip()
    from oracle import bopt as BO
    from oracle import nfft as NF
    from oracle import windows as W
    from paper_2302_00414_gb300 import api
    x = inputs.random_points(N, d, 3 + d)
    p = L.Plan(x, M, 2.0, m, prec)
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    nd = np.complex64 if prec == "fp32" else np.complex128
    md = {"plain": L.MODE_PLAIN, "dcf": L.MODE_DCF, "bopt": L.MODE_BOPT}[mode]
    w = np.ones(N)
    coef = None
    if mode == "dcf":
        w = inputs.coeffs_complex((N,), 4) / N
        p.set_weights(w)
    elif mode == "bopt":
        p.optimize_B()
        coef = p.get_bopt()
    tol_gpu = 1e-5 if prec == "fp32" else 1e-12
    tol_oracle = 1e-5 if prec == "fp32" else 1e-9
    for call in range(2):
        f_np = inputs.samples_complex(N, 10 + call).astype(nd)
        f = to_dev(torch, f_np)
        ref = p.adjoint(f, mode=md)
        out = torch.full((M,) * d, float("nan"), dtype=cd, device="cuda")
        s = api.infft_adjoint_noalloc(p.handle, md, f.data_ptr(), out.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        assert s == L.OK, L.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().ravel()
        assert rel(got, ref.cpu().numpy()) <= tol_gpu
        c = f_np.astype(np.complex128)
        if mode == "bopt":
            orc = BO.reconstruct(x, c, coef, M, 2.0, m, W.KB, BO.PATTERN_2M2)
        else:
            orc = NF.adjoint_nfft(x, w * c, M, 2.0, m)
        assert rel(got, orc) <= tol_oracle


def test_noalloc_rejects_oversized_plan_and_host_buffers():
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300 import api
    x = inputs.random_points(1000, 2, 5)
    big = L.Plan(x, 2048, 2.0, 4, "fp32")   # 4096^2 grid: > 32 MiB of scratch
    f = to_dev(torch, inputs.samples_complex(1000, 6), torch.complex64)
    out = torch.empty((2048, 2048), dtype=torch.complex64, device="cuda")
    s = api.infft_adjoint_noalloc(big.handle, L.MODE_PLAIN, f.data_ptr(), out.data_ptr(), 0)
    assert s == L.EINVAL and "scratch" in L.last_error()
    small = L.Plan(x, 16, 2.0, 4, "fp32")
    h = np.zeros((16, 16), dtype=np.complex64)
    s = api.infft_adjoint_noalloc(small.handle, L.MODE_PLAIN, f.data_ptr(), h.ctypes.data, 0)
    assert s == L.EINVAL and "device pointers" in L.last_error()


def test_noalloc_mode_errors_match_adjoint():
    """Misuse gives the same status codes as infft_adjoint."""
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300 import api
    x = inputs.random_points(500, 2, 8)
    f = to_dev(torch, inputs.samples_complex(500, 9), torch.complex128)
    out = torch.empty((16, 16), dtype=torch.complex128, device="cuda")
    dirichlet = L.Plan(x, 16, 2.0, 3, "fp64", window="dirichlet")
    kb = L.Plan(x, 16, 2.0, 3, "fp64")
    for plan, mode in ((dirichlet, L.MODE_PLAIN), (kb, L.MODE_DCF), (kb, L.MODE_BOPT), (kb, 7)):
        a = api.infft_adjoint(plan.handle, mode, f.data_ptr(), out.data_ptr(), 0)
        b = api.infft_adjoint_noalloc(plan.handle, mode, f.data_ptr(), out.data_ptr(), 0)
        assert a == b and a != L.OK
