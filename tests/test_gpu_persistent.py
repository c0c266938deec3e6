"""The persistent batched d = 2 adjoint (Algorithm 3.7 / 2.4 over many point sets in one
launch) against the staged kernels (spread, merging pass along x, pass along y as separate
launches): every sum is formed in the same order, so the results are bitwise equal.  Also
against the FP64 oracle's Algorithm 2.4, in graph replays, with one plan in several scratch
slots, with two batches in flight on two streams, and with no bounded wait giving up."""
import numpy as np
import pytest

import inputs
from oracle import nfft as NF
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu


def _sets(specs, seed):
    out = []
    for i, (M, N) in enumerate(specs):
        x = inputs.random_points(N, 2, seed + i)
        f = inputs.samples_complex(N, seed + 100 + i)
        w = inputs.rng(seed + 200 + i).uniform(0.5, 1.5, N) / N
        out.append((M, x, f, w))
    return out


def _run(L, torch, plans, fs, mode, monkeypatch, form):
    monkeypatch.setenv("INFFT_PERSISTENT", form)
    hs = [torch.empty((p.M, p.M), dtype=torch.complex64, device="cuda") for p in plans]
    L.adjoint_batched(plans, fs, hs, mode)
    torch.cuda.synchronize()
    return [h.cpu().numpy() for h in hs]


@pytest.mark.parametrize("m", [2, 3, 4])
@pytest.mark.parametrize("mode", ["plain", "dcf"])
@pytest.mark.parametrize("tile", [0, 8])
def test_persistent_batch_equals_staged_kernels(m, mode, tile, monkeypatch):
    L, torch = lib_or_skip()
    if tile and 2 * m > tile:
        pytest.skip("the register-row path needs 2m <= T")
    specs = [(8, 150), (16, 1), (32, 4000), (64, 20000), (128, 70000), (32, 33), (64, 3000), (16, 900)]
    sets = _sets(specs, 900 + m)
    tune = {"tile": tile} if tile else None
    plans, fs = [], []
    for M, x, f, w in sets:
        p = L.Plan(x, M, 2.0, m, "fp32", tune=tune)
        if mode == "dcf":
            p.set_weights(w.astype(np.complex128))
        plans.append(p)
        fs.append(to_dev(torch, f, torch.complex64))
    md = L.MODE_DCF if mode == "dcf" else L.MODE_PLAIN
    t0 = L.wait_timeouts()
    staged = _run(L, torch, plans, fs, md, monkeypatch, "0")
    pers = _run(L, torch, plans, fs, md, monkeypatch, "1")
    again = _run(L, torch, plans, fs, md, monkeypatch, "1")
    assert L.wait_timeouts() == t0
    for a, b, c in zip(staged, pers, again):
        assert np.array_equal(a, b)
        assert np.array_equal(b, c)
    M, x, f, w = sets[4]
    c = f.astype(np.complex64).astype(np.complex128) * (w if mode == "dcf" else 1.0)
    assert rel(pers[4], NF.adjoint_nfft(x, c, M, 2.0, m)) < 1e-5


def test_persistent_graph_slots_and_single_calls(monkeypatch):
    """A graph replay of the persistent batch, a plan appearing three times (three scratch
    slots, so three sets of counters), and single calls (a batch of one) give the staged
    results bit for bit."""
    L, torch = lib_or_skip()
    sets = _sets([(64, 15000), (128, 50000), (32, 3000)], 950)
    plans, fs = [], []
    for M, x, f, w in sets:
        p = L.Plan(x, M, 2.0, 4, "fp32")
        p.set_weights(w.astype(np.complex128))
        plans.append(p)
        fs.append(to_dev(torch, f, torch.complex64))
    extra = [to_dev(torch, inputs.samples_complex(15000, 960 + k), torch.complex64) for k in range(2)]
    P = plans + [plans[0], plans[0]]
    F = fs + extra
    t0 = L.wait_timeouts()
    staged = _run(L, torch, P, F, L.MODE_DCF, monkeypatch, "0")
    pers = _run(L, torch, P, F, L.MODE_DCF, monkeypatch, "1")
    for a, b in zip(staged, pers):
        assert np.array_equal(a, b)
    monkeypatch.setenv("INFFT_PERSISTENT", "1")
    hs = [torch.empty((p.M, p.M), dtype=torch.complex64, device="cuda") for p in P]
    b = L.Batch(P, F, hs, L.MODE_DCF)
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    for h, a in zip(hs, staged):
        assert np.array_equal(h.cpu().numpy(), a)
    b.close()
    for p, f, a in zip(plans, fs, staged):
        assert np.array_equal(p.adjoint(f, mode=L.MODE_DCF).cpu().numpy(), a)
    assert L.wait_timeouts() == t0


def test_two_persistent_batches_in_flight(monkeypatch):
    """Two batches on two streams at once (as the server issues them), each a persistent
    launch with its own jobs' counters, give the results of running them one at a time."""
    L, torch = lib_or_skip()
    A = _sets([(64, 12000), (32, 2500), (128, 40000)], 970)
    B = _sets([(128, 45000), (64, 9000)], 980)
    def build(sets):
        plans, fs = [], []
        for M, x, f, w in sets:
            p = L.Plan(x, M, 2.0, 4, "fp32")
            p.set_weights(w.astype(np.complex128))
            plans.append(p)
            fs.append(to_dev(torch, f, torch.complex64))
        return plans, fs
    pa, fa = build(A)
    pb, fb = build(B)
    ra = _run(L, torch, pa, fa, L.MODE_DCF, monkeypatch, "0")
    rb = _run(L, torch, pb, fb, L.MODE_DCF, monkeypatch, "0")
    monkeypatch.setenv("INFFT_PERSISTENT", "1")
    t0 = L.wait_timeouts()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ha = [torch.empty((p.M, p.M), dtype=torch.complex64, device="cuda") for p in pa]
    hb = [torch.empty((p.M, p.M), dtype=torch.complex64, device="cuda") for p in pb]
    torch.cuda.synchronize()
    for _ in range(4):
        L.adjoint_batched(pa, fa, ha, L.MODE_DCF, stream=s1)
        L.adjoint_batched(pb, fb, hb, L.MODE_DCF, stream=s2)
    torch.cuda.synchronize()
    assert L.wait_timeouts() == t0
    for h, a in zip(ha, ra):
        assert np.array_equal(h.cpu().numpy(), a)
    for h, a in zip(hb, rb):
        assert np.array_equal(h.cpu().numpy(), a)
