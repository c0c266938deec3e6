"""Repeated plans in one batched call, and the continuous-batching loop, on the GPU.

Every reconstruction h = D^* F^* B^* W f (Algorithm 3.7) returned by a batch or by the
serving loop must be bitwise equal to the same reconstruction computed alone: a job's
arithmetic does not depend on the batch it runs in, on the stream, or on the scratch
set it uses.
"""
import numpy as np
import pytest

import inputs
from tests.gpu_util import lib_or_skip, to_dev

pytestmark = pytest.mark.gpu


def test_repeated_plan_in_batch_bitwise():
    L, torch = lib_or_skip()
    x = inputs.random_points(20000, 2, 5)
    y = inputs.polar(64, 48)
    p = L.Plan(x, 64, 2.0, 4, "fp32")
    q = L.Plan(y, 32, 2.0, 4, "fp32")
    for pl in (p, q):
        pl.weights(max_iter=20)
    plans = [p, q, p, p, q]
    fs = [to_dev(torch, inputs.samples_complex(pl.N, 10 + i), torch.complex64) for i, pl in enumerate(plans)]
    alone = [pl.adjoint(f, mode=L.MODE_DCF).clone() for pl, f in zip(plans, fs)]
    before = p.device_bytes
    outs = [torch.empty_like(a) for a in alone]
    L.adjoint_batched(plans, fs, outs, L.MODE_DCF)
    torch.cuda.synchronize()
    for a, b in zip(alone, outs):
        assert torch.equal(a, b)
    assert p.device_bytes > before            # two extra scratch sets for p
    grown = p.device_bytes
    outs2 = [torch.zeros_like(a) for a in alone]
    b = L.Batch(plans, fs, outs2, L.MODE_DCF)
    for _ in range(2):
        b.run()
    torch.cuda.synchronize()
    for a, o in zip(alone, outs2):
        assert torch.equal(a, o)
    assert p.device_bytes == grown            # scratch sets are kept and reused
    b.close()
    # caller-chosen scratch sets, two batches of the same plans in flight on two streams
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs3 = [torch.zeros_like(a) for a in alone]
    outs4 = [torch.zeros_like(a) for a in alone]
    torch.cuda.synchronize()
    L.adjoint_batched(plans, fs, outs3, L.MODE_DCF, stream=s1.cuda_stream, slots=[0, 0, 1, 2, 1])
    L.adjoint_batched(plans, fs, outs4, L.MODE_DCF, stream=s2.cuda_stream, slots=[3, 2, 4, 5, 3])
    torch.cuda.synchronize()
    for a, o3, o4 in zip(alone, outs3, outs4):
        assert torch.equal(a, o3) and torch.equal(a, o4)
    for bad in ([0, 0, 0, 1, 1], [0, 0, 1, -1, 1], [0, 0, 1, 2, 2000]):
        with pytest.raises(L.InfftError):
            L.adjoint_batched(plans, fs, outs3, L.MODE_DCF, slots=bad)
    # host buffers are staged through the plan's I/O buffers: no repeats
    fh = [inputs.samples_complex(p.N, 1).astype(np.complex64) for _ in range(2)]
    hh = [np.empty((64, 64), np.complex64) for _ in range(2)]
    with pytest.raises(L.InfftError):
        L.adjoint_batched([p, p], fh, hh, L.MODE_DCF)


def test_serving_loop_results_match_alone():
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300.serve import Backend, PointSet, Request, Server, latency_summary
    sets = [PointSet(0, 2, 128, inputs.random_points(60000, 2, 1)),
            PointSet(1, 2, 64, inputs.polar(128, 96)),
            PointSet(2, 3, 16, inputs.random_points(8000, 3, 3)),
            PointSet(3, 2, 128, inputs.jittered_grid(200, 2, 4))]
    server = Server(Backend(weights_iters=10), max_batch=16, streams=3, max_repeat=4)
    for ps in sets:
        server.register(ps)
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(240):
        k = int(rng.choice(4, p=[0.55, 0.2, 0.1, 0.15]))
        f = to_dev(torch, inputs.samples_complex(sets[k].x.shape[0], 1000 + i), torch.complex64)
        reqs.append(Request(rid=i, key=k, f=f))
    for r in reqs[:120]:            # a burst, then the rest while the first batches run
        server.submit(r)
    for _ in range(5):
        server.step()
    for r in reqs[120:]:
        server.submit(r)
    server.drain(timeout=300)
    torch.cuda.synchronize()
    done = {r.rid: r for r in server.completed}
    assert sorted(done) == list(range(240))
    for r in reqs:
        ref = server.plans[r.key].adjoint(r.f, mode=L.MODE_DCF)
        assert torch.equal(ref, done[r.rid].out), r.rid
    summ = latency_summary(server.completed)
    assert summ["mean_batch"] > 1
    assert server.stats["max_inflight"] > 1
    assert server.stats["new_sets"] == 4
    server.close()


def test_serving_loop_evicts_under_budget():
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300.serve import Backend, PointSet, Request, Server
    be = Backend(weights_iters=5)
    sets = [PointSet(k, 2, 32, inputs.random_points(3000, 2, 20 + k)) for k in range(4)]
    need = max(be.estimate_bytes(ps) for ps in sets)
    probe = be.build_plan(sets[0], torch.cuda.current_stream())
    actual = be.plan_bytes(probe)
    be.release(probe)
    # room for one resident plan and one being built, not for two resident plans and a build
    budget = int(need + 1.5 * actual)
    server = Server(be, mem_budget=budget, max_batch=8, streams=2)
    for ps in sets:
        server.register(ps)
    fs = {}
    for i in range(16):
        k = i % 4
        fs[i] = to_dev(torch, inputs.samples_complex(3000, 50 + i), torch.complex64)
        server.submit(Request(rid=i, key=k, f=fs[i]))
        server.drain(timeout=120)
    assert len(server.completed) == 16
    assert server.stats["evicted"] > 0
    assert server.resident_bytes <= budget
    # results equal a fresh plan on the same points with the same weights
    for r in server.completed[-4:]:
        pl = server.plans.get(r.key)
        if pl is None:
            continue
        assert torch.equal(pl.adjoint(r.f, mode=L.MODE_DCF), r.out)
    server.close()


def test_pooled_plans_give_the_same_results():
    """Plans whose memory comes from the library's stream-ordered pool compute bit for bit
    what ordinary plans compute: weights (Toeplitz CG), DCF reconstruction through host and
    device buffers, repeated plans in a batch, B_opt and the inverse adjoint."""
    L, torch = lib_or_skip()
    x = inputs.random_points(5000, 2, 61)
    s = torch.cuda.Stream()
    res = []
    for pooled in (False, True):
        p = L.Plan(x, 32, 2.0, 4, "fp64", stream=s.cuda_stream, pooled=pooled)
        p.weights(max_iter=50, stream=s.cuda_stream)
        f = inputs.samples_complex(p.N, 62)
        fd = to_dev(torch, f)
        hd = to_dev(torch, inputs.coeffs_complex((32, 32), 63))
        torch.cuda.synchronize()        # the copies above ran on the default stream
        h_dev = p.adjoint(fd, mode=L.MODE_DCF, stream=s.cuda_stream)
        h_host = p.adjoint(f, mode=L.MODE_DCF)
        with torch.cuda.stream(s):
            outs = [torch.empty((32, 32), dtype=torch.complex128, device="cuda") for _ in range(3)]
            L.adjoint_batched([p, p, p], [fd, fd, fd], outs, L.MODE_DCF, stream=s.cuda_stream, slots=[0, 2, 1])
        p.optimize_B(stream=s.cuda_stream)
        g = p.inverse_adjoint(hd, stream=s.cuda_stream)
        s.synchronize()
        res.append([p.get_weights(), h_dev.cpu().numpy(), h_host] + [o.cpu().numpy() for o in outs] +
                   [g.cpu().numpy()])
        p.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)
