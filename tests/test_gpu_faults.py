"""Failure detection without a GPU fault: host-side injected failures (infft_inject_faults)
come back as status codes, leave the library usable, and the serving loop fails only the
requests they concern."""
import numpy as np
import pytest

import inputs
from tests.gpu_util import lib_or_skip, to_dev

pytestmark = pytest.mark.gpu


def test_injected_failures_are_reported_and_recovered():
    L, torch = lib_or_skip()
    x = inputs.random_points(3000, 2, 81)
    f = to_dev(torch, inputs.samples_complex(3000, 82), torch.complex64)
    p = L.Plan(x, 32, 2.0, 4, "fp32")
    p.weights(max_iter=20)
    h_ref = p.adjoint(f, mode=L.MODE_DCF).clone()
    try:
        L.inject_faults(1)                          # allocations fail
        with pytest.raises(L.InfftError) as e:
            L.Plan(x, 32, 2.0, 4, "fp32")
        assert e.value.status == 2                  # INFFT_ENOMEM
        L.inject_faults(2)                          # launches report failure
        with pytest.raises(L.InfftError) as e:
            p.adjoint(f, mode=L.MODE_DCF)
        assert e.value.status == 3                  # INFFT_ECUDA
        torch.cuda.synchronize()                    # the queued kernels still ran cleanly
        L.inject_faults(4)                          # the CG does not converge
        info = p.weights(max_iter=20)
        assert info["status"] == 4                  # INFFT_ENOTCONV, weights stored
    finally:
        L.inject_faults(0)
    assert torch.equal(p.adjoint(f, mode=L.MODE_DCF), h_ref)
    q = L.Plan(x, 32, 2.0, 4, "fp32")
    assert q.device_bytes > 0


def test_serving_loop_survives_failed_builds():
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300.serve import Backend, PointSet, Request, Server
    sets = [PointSet(k, 2, 32, inputs.random_points(2000, 2, 90 + k)) for k in range(3)]
    server = Server(Backend(weights_iters=5), max_batch=8, streams=2)
    for ps in sets:
        server.register(ps)
    fs = [to_dev(torch, inputs.samples_complex(2000, 95 + k), torch.complex64) for k in range(3)]
    server.submit(Request(rid=0, key=0, f=fs[0]))
    server.drain(timeout=120)
    try:
        L.inject_faults(1)
        server.submit(Request(rid=1, key=1, f=fs[1]))   # its build fails
        server.drain(timeout=120)
    finally:
        L.inject_faults(0)
    server.submit(Request(rid=2, key=2, f=fs[2]))
    server.submit(Request(rid=3, key=0, f=fs[0]))
    server.drain(timeout=120)
    assert [r.rid for r in server.failed] == [1]
    assert isinstance(server.failed[0].error, L.InfftError)
    assert sorted(r.rid for r in server.completed) == [0, 2, 3]
    assert server.stats["failed_sets"] == 1
    server.close()
