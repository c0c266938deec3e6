"""Full-size workloads on the GPU, checked on sampled coefficients against the FP64
oracle's exact sums with the same weights (the hot-path parity of Algorithm 3.7).

* polar grid, d=2, M=128, 512 angles x 256 radii (N = 131072), FP32 spreading with m=4
  and m=6, weights from the float64 CG at degree 2M (iterations capped: the polar
  system is ill-conditioned, so only the residual is recorded);
* stack of spirals, d=3, M=64, 64 planes x 32768 points (N = 2^21), FP32, m=4;
* a batch of random sets up to M=256 executed through one CUDA graph.
Exactness cannot hold on these grids, so the checks are parity with the oracle at the
FP32 bound (1e-5) and finiteness / monotonicity of the CG residual.
"""
import numpy as np
import pytest

import inputs
from oracle import fourier as FO
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu


def sampled_parity(x, w, f, M, d, h, nk, seed):
    K = M ** d
    ks = np.random.default_rng(seed).choice(K, size=min(nk, K), replace=False)
    ref = FO.adjoint_ndft(x, w * f, M, k_subset=ks)
    return rel(h.ravel()[ks], ref)


@pytest.mark.parametrize("m", [4, 6])
def test_polar_d2_M128(m):
    L, torch = lib_or_skip()
    x = inputs.polar(512, 256)
    M = 128
    p = L.Plan(x, M, 2.0, m, "fp32")
    info = p.weights(max_iter=30, rel_tol=1e-13)
    assert np.isfinite(info["residual_inf"])
    w = p.get_weights()
    assert np.all(np.isfinite(w))
    f = inputs.samples_complex(x.shape[0], 3)
    h = p.adjoint(to_dev(torch, f, torch.complex64), mode=L.MODE_DCF).cpu().numpy()
    assert sampled_parity(x, w, f, M, 2, h, 256, 4) < 1e-5


def test_spiral_stack_d3_M64():
    L, torch = lib_or_skip()
    x = inputs.spiral_stack(64, 32768, 64)
    M = 64
    p = L.Plan(x, M, 2.0, 4, "fp32")
    info = p.weights(max_iter=8, rel_tol=1e-13)
    assert np.isfinite(info["residual_inf"])
    w = p.get_weights()
    f = inputs.samples_complex(x.shape[0], 5)
    h = p.adjoint(to_dev(torch, f, torch.complex64), mode=L.MODE_DCF).cpu().numpy()
    assert sampled_parity(x, w, f, M, 3, h, 48, 6) < 1e-5


def test_batched_graph_large_sets():
    L, torch = lib_or_skip()
    sets = inputs.batch_sets(6, 21)
    sets[0] = (256, inputs.random_points(5 * 256 * 256, 2, 77))
    plans, fs, hs, ws, fh = [], [], [], [], []
    for i, (M, x) in enumerate(sets):
        p = L.Plan(x, M, 2.0, 4, "fp32")
        w = inputs.coeffs_complex((x.shape[0],), 300 + i) / x.shape[0]
        p.set_weights(w)
        f = inputs.samples_complex(x.shape[0], 400 + i)
        plans.append(p)
        ws.append(w)
        fh.append(f)
        fs.append(to_dev(torch, f, torch.complex64))
        hs.append(torch.zeros((M, M), dtype=torch.complex64, device="cuda"))
    b = L.Batch(plans, fs, hs, L.MODE_DCF)
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    for i, (M, x) in enumerate(sets):
        assert sampled_parity(x, ws[i], fh[i], M, 2, hs[i].cpu().numpy(), 128, 500 + i) < 1e-5


def test_graph_batch_over_pinned_host_buffers():
    """A graph batch whose samples and results live in page-locked host memory holds the
    copies too: every replay gives the device-buffer result bit for bit; pageable host
    buffers are refused."""
    L, torch = lib_or_skip()
    sets = inputs.batch_sets(5, 31)
    plans, fd, hd, fh, hh = [], [], [], [], []
    for i, (M, x) in enumerate(sets):
        p = L.Plan(x, M, 2.0, 4, "fp32")
        p.set_weights(inputs.coeffs_complex((x.shape[0],), 40 + i) / x.shape[0])
        plans.append(p)
        f = torch.from_numpy(inputs.samples_complex(x.shape[0], 50 + i).astype(np.complex64))
        fd.append(f.cuda())
        hd.append(torch.empty((M, M), dtype=torch.complex64, device="cuda"))
        fh.append(f.pin_memory())
        hh.append(torch.zeros((M, M), dtype=torch.complex64).pin_memory())
    L.Batch(plans, fd, hd, L.MODE_DCF).run()
    torch.cuda.synchronize()
    hb = L.Batch(plans, [t.numpy() for t in fh], [t.numpy() for t in hh], L.MODE_DCF)
    for rep in range(3):
        for t in hh:
            t.zero_()
        hb.run()
        torch.cuda.synchronize()
        for a, b in zip(hh, hd):
            assert np.array_equal(a.numpy(), b.cpu().numpy())
    # the samples and results as slices of one page-locked allocation each: the graph copies
    # adjacent ranges at once; same results
    nf = [int(t.numel()) for t in fh]
    nh = [M * M for M, _ in sets]
    fa = torch.empty(sum(nf), dtype=torch.complex64).pin_memory()
    ha = torch.zeros(sum(nh), dtype=torch.complex64).pin_memory()
    of, oh = np.cumsum([0] + nf), np.cumsum([0] + nh)
    fs2 = [fa[of[i]:of[i + 1]] for i in range(len(sets))]
    for a, t in zip(fs2, fh):
        a.copy_(t)
    hs2 = [ha[oh[i]:oh[i + 1]].view(M, M) for i, (M, _) in enumerate(sets)]
    hb2 = L.Batch(plans, [t.numpy() for t in fs2], [t.numpy() for t in hs2], L.MODE_DCF)
    for rep in range(2):
        ha.zero_()
        hb2.run()
        torch.cuda.synchronize()
        for a, b in zip(hs2, hd):
            assert np.array_equal(a.numpy(), b.cpu().numpy())
    pageable = [np.zeros((M, M), dtype=np.complex64) for M, _ in sets]
    with pytest.raises(L.InfftError):
        L.Batch(plans, [t.numpy() for t in fh], pageable, L.MODE_DCF)
