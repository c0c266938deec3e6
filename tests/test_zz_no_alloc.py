"""The allocation-free reconstruction entry point, infft_adjoint_noalloc.

Some callers cannot allocate device memory during a call (an external allocator
owns the device memory, or cudaMalloc's synchronisation is not acceptable in their
loop).  infft_adjoint_noalloc serves them from a fixed scratch array inside the
library.  This file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.  It also passes in a
fresh process on its own.
"""
import numpy as np
import pytest

import inputs
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,mode", [("fp32", "dcf"), ("fp64", "plain")])
def test_noalloc_matches_adjoint_two_calls(prec, mode):
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300 import api
    x = inputs.random_points(20000, 2, 3)
    M = 64
    p = L.Plan(x, M, 2.0, 4, prec)
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    md = L.MODE_PLAIN
    if mode == "dcf":
        p.set_weights(inputs.coeffs_complex((20000,), 4) / 20000)
        md = L.MODE_DCF
    tol = 1e-5 if prec == "fp32" else 1e-12
    for call in range(2):  # the scratch keeps the previous call's contents
        f = to_dev(torch, inputs.samples_complex(20000, 10 + call), cd)
        ref = p.adjoint(f, mode=md)
        out = torch.full((M, M), float("nan"), dtype=cd, device="cuda")
        s = api.infft_adjoint_noalloc(p.handle, md, f.data_ptr(), out.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        assert s == L.OK, L.last_error()
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= tol


def test_noalloc_rejects_oversized_plan_and_host_buffers():
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300 import api
    x = inputs.random_points(1000, 2, 5)
    big = L.Plan(x, 2048, 2.0, 4, "fp32")   # 4096^2 grid: > 32 MiB of scratch
    f = to_dev(torch, inputs.samples_complex(1000, 6), torch.complex64)
    out = torch.empty((2048, 2048), dtype=torch.complex64, device="cuda")
    s = api.infft_adjoint_noalloc(big.handle, L.MODE_PLAIN, f.data_ptr(), out.data_ptr(), 0)
    assert s == 1 and "scratch" in L.last_error()
    small = L.Plan(x, 16, 2.0, 4, "fp32")
    h = np.zeros((16, 16), dtype=np.complex64)
    s = api.infft_adjoint_noalloc(small.handle, L.MODE_PLAIN, f.data_ptr(), h.ctypes.data, 0)
    assert s == 1 and "device pointers" in L.last_error()
