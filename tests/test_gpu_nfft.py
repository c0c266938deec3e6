"""Parity of the CUDA adjoint NFFT / NFFT (Algorithms 2.4 / 2.1) with the FP64 oracle.

FP64 plans run the same algorithm as the oracle's Algorithm 2.4 / 2.1, so they
are compared with it at 1e-12.  FP32 plans are compared with the exact sums
(eq. nfft*, eq. nfft) at the 1e-5 relative l2 bound required for FP32
spreading, and with the oracle's Algorithm 2.4 at a bound derived from float32
rounding (1e-5 as well).  Sizes span several tiles and ragged tails.
"""
import numpy as np
import pytest

import inputs
from oracle import fourier as FO
from oracle import bopt as BO
from oracle import nfft as NF
from tests.gpu_util import lib_or_skip, rel, to_dev

pytestmark = pytest.mark.gpu


def kb_bound(m, sigma):
    """Kaiser-Bessel error estimate of the cited window literature (see test_oracle_nfft)."""
    s = np.sqrt(1 - 1 / sigma)
    return 4 * np.pi * (np.sqrt(m) + m) * s ** 0.5 * np.exp(-2 * np.pi * m * s)

CASES = [  # d, M, N, sigma, m, generator
    (1, 64, 256, 2.0, 6, "jitter"),
    (1, 128, 1001, 2.0, 4, "random"),
    (2, 32, 3000, 2.0, 4, "random"),
    (2, 64, 9001, 2.0, 6, "random"),
    (2, 16, 200, 2.0, 2, "random"),
    (2, 64, 4096, 2.0, 4, "polar"),
    (2, 8, 50, 2.0, 3, "random"),
    (3, 16, 2000, 2.0, 3, "random"),
    (3, 8, 700, 2.0, 2, "random"),
    (3, 16, 2500, 2.0, 4, "random"),
    (3, 16, 2500, 2.0, 5, "random"),
    (3, 8, 4000, 2.0, 3, "clustered"),
    (2, 32, 3000, 2.0, 4, "clustered"),
]


def points(d, N, gen, seed):
    if gen == "jitter":
        return inputs.jittered_1d(N, seed)
    if gen == "clustered":   # many points per base cell, some exactly repeated
        g = inputs.rng(seed)
        centres = g.uniform(-0.5, 0.5, size=(7, d))
        x = centres[g.integers(0, 7, size=N)] + g.uniform(-1e-3, 1e-3, size=(N, d))
        x[: N // 4] = centres[0]
        return x
    if gen == "polar":
        n = int(np.sqrt(N))
        return inputs.polar(n, n)
    return inputs.random_points(N, d, seed)


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}M{c[1]}N{c[2]}m{c[4]}{c[5]}" for c in CASES])
def test_adjoint_fp64_matches_oracle_algorithm(case):
    L, torch = lib_or_skip()
    d, M, N, sigma, m, gen = case
    x = points(d, N, gen, 1)
    N = x.shape[0]
    f = inputs.samples_complex(N, 2)
    ref = NF.adjoint_nfft(x, f, M, sigma, m)
    p = L.Plan(x, M, sigma, m, "fp64")
    h = p.adjoint(to_dev(torch, f)).cpu().numpy().ravel()
    assert rel(h, ref) < 1e-12


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}M{c[1]}N{c[2]}m{c[4]}{c[5]}" for c in CASES])
def test_forward_fp64_matches_oracle_algorithm(case):
    L, torch = lib_or_skip()
    d, M, N, sigma, m, gen = case
    x = points(d, N, gen, 3)
    fh = inputs.coeffs_complex((M,) * d, 4)
    ref = NF.nfft(x, fh, M, sigma, m)
    p = L.Plan(x, M, sigma, m, "fp64")
    f = p.forward(to_dev(torch, fh)).cpu().numpy()
    assert rel(f, ref) < 1e-12


@pytest.mark.parametrize("d,M,N,m", [(1, 64, 256, 6), (2, 64, 9001, 6), (2, 64, 9001, 4), (2, 128, 20000, 4),
                                     (3, 16, 3000, 4), (3, 16, 3000, 6), (3, 32, 30000, 4)])
def test_fp32_within_1e5_of_exact_sums(d, M, N, m):
    L, torch = lib_or_skip()
    x = inputs.random_points(N, d, 5)
    f = inputs.samples_complex(N, 6)
    p = L.Plan(x, M, 2.0, m, "fp32")
    h = p.adjoint(to_dev(torch, f, torch.complex64)).cpu().numpy()
    assert rel(h, FO.adjoint_ndft(x, f, M)) < 1e-5
    fh = inputs.coeffs_complex((M,) * d, 7)
    fx = p.forward(to_dev(torch, fh, torch.complex64)).cpu().numpy()
    assert rel(fx, FO.ndft(x, fh, M)) < 1e-5


def test_edge_points_and_single_point():
    L, torch = lib_or_skip()
    M, sigma, m = 16, 2.0, 4
    # points on the boundary of the torus, below -1/2, on grid nodes, duplicates
    x = np.array([[-0.5, -0.5], [0.5 - 1e-12, 0.25], [-0.5 - 1e-3, 0.0], [0.0, 0.0], [0.0, 0.0],
                  [1.0 / 32, -3.0 / 32], [0.49999, -0.49999]])
    f = inputs.samples_complex(len(x), 8)
    p = L.Plan(x, M, sigma, m, "fp64")
    h = p.adjoint(to_dev(torch, f)).cpu().numpy()
    assert rel(h, NF.adjoint_nfft(x, f, M, sigma, m)) < 1e-12
    # N = 1
    x1 = np.array([[0.3141, -0.2718]])
    p1 = L.Plan(x1, M, sigma, m, "fp64")
    h1 = p1.adjoint(to_dev(torch, np.array([1.0 + 0j]))).cpu().numpy().ravel()
    K = FO.index_set(M, 2)
    assert np.max(np.abs(h1 - np.exp(-2j * np.pi * (K @ x1[0])))) < kb_bound(m, sigma)


def test_host_buffers_equal_device_buffers():
    L, torch = lib_or_skip()
    x = inputs.random_points(5000, 2, 9)
    f = inputs.samples_complex(5000, 10).astype(np.complex64)
    p = L.Plan(x, 64, 2.0, 4, "fp32")
    hd = p.adjoint(to_dev(torch, f)).cpu().numpy()
    hh = p.adjoint(f)  # numpy in, numpy out: staged by the library
    assert np.array_equal(hd, hh)


def test_deterministic_bitwise():
    L, torch = lib_or_skip()
    x = inputs.polar(128, 64)
    f = to_dev(torch, inputs.samples_complex(x.shape[0], 11), torch.complex64)
    p = L.Plan(x, 64, 2.0, 4, "fp32")
    a = p.adjoint(f).cpu().numpy()
    b = p.adjoint(f).cpu().numpy()
    q = L.Plan(x, 64, 2.0, 4, "fp32")
    c = q.adjoint(f).cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_batched_and_graph_equal_single_calls():
    L, torch = lib_or_skip()
    sets = inputs.batch_sets(6, 12, Ms=(16, 32, 64))
    plans, fs, outs, singles = [], [], [], []
    for i, (M, x) in enumerate(sets):
        p = L.Plan(x, M, 2.0, 4, "fp32")
        f = to_dev(torch, inputs.samples_complex(x.shape[0], 100 + i), torch.complex64)
        plans.append(p)
        fs.append(f)
        outs.append(torch.empty((M, M), dtype=torch.complex64, device="cuda"))
        singles.append(p.adjoint(f).cpu().numpy())
    L.adjoint_batched(plans, fs, outs)
    for o, s in zip(outs, singles):
        assert np.array_equal(o.cpu().numpy(), s)
    g_outs = [torch.zeros_like(o) for o in outs]
    b = L.Batch(plans, fs, g_outs)
    b.run()
    torch.cuda.synchronize()
    for o, s in zip(g_outs, singles):
        assert np.array_equal(o.cpu().numpy(), s)


def test_error_codes():
    L, torch = lib_or_skip()
    x = inputs.random_points(100, 2, 13)
    with pytest.raises(L.InfftError) as e:
        L.Plan(x, 15, 2.0, 4)
    assert e.value.status == 1  # EINVAL: M odd
    with pytest.raises(L.InfftError) as e:
        L.Plan(x, 12, 2.0, 4)
    assert e.value.status == 7  # EUNSUPPORTED: M_sigma = 24
    with pytest.raises(L.InfftError) as e:
        L.Plan(x, 4, 2.0, 4)
    assert e.value.status == 1  # 2m+2 > M_sigma
    p = L.Plan(x, 16, 2.0, 4)
    f = to_dev(torch, inputs.samples_complex(100, 1), torch.complex64)
    with pytest.raises(L.InfftError) as e:
        p.adjoint(f, mode=L.MODE_DCF)
    assert e.value.status == 6  # ESTATE: no weights yet


def test_batched_page_locked_host_buffers():
    """Page-locked host inputs and outputs (gathered and scattered by the library's copy
    kernel), pageable ones (cudaMemcpyAsync) and device buffers give the same bits."""
    L, torch = lib_or_skip()
    sets = inputs.batch_sets(5, 31)
    plans, fd, hd, fp, hp, fn, hn = [], [], [], [], [], [], []
    for i, (M, x) in enumerate(sets):
        p = L.Plan(x, M, 2.0, 4, "fp32")
        p.set_weights(inputs.coeffs_complex((x.shape[0],), 700 + i) / x.shape[0])
        f = inputs.samples_complex(x.shape[0], 710 + i).astype(np.complex64)
        plans.append(p)
        fd.append(to_dev(torch, f))
        hd.append(torch.empty((M, M), dtype=torch.complex64, device="cuda"))
        fp.append(torch.from_numpy(f).pin_memory())
        hp.append(torch.empty((M, M), dtype=torch.complex64).pin_memory())
        fn.append(f)
        hn.append(np.empty((M, M), np.complex64))
    L.adjoint_batched(plans, fd, hd, L.MODE_DCF)
    torch.cuda.synchronize()
    L.adjoint_batched(plans, fp, hp, L.MODE_DCF)
    L.adjoint_batched(plans, fn, hn, L.MODE_DCF)
    for a, b, c in zip(hd, hp, hn):
        assert np.array_equal(a.cpu().numpy(), b.numpy())
        assert np.array_equal(a.cpu().numpy(), c)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", ["plain", "dcf"])
def test_spread2d_prefetch_forms_equal(prec, mode, monkeypatch):
    """The d = 2 spread with the next points' data prefetched (chosen for small grids) and
    the one without (large grids) make the same sums in the same order: equal bit for bit,
    and both within the bounds of the oracle's Algorithm 2.4."""
    L, torch = lib_or_skip()
    M, sigma, m = 64, 2.0, 4
    x = inputs.random_points(9001, 2, 21)
    f = inputs.samples_complex(len(x), 22)
    w = inputs.rng(23).uniform(0.5, 1.5, len(x)) / len(x)
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    p = L.Plan(x, M, sigma, m, prec)
    md = L.MODE_PLAIN
    if mode == "dcf":
        p.set_weights(w.astype(np.complex128))
        md = L.MODE_DCF
    fd = to_dev(torch, f, cdt)
    out = {}
    for form in ("0", "1"):
        monkeypatch.setenv("INFFT_SPREAD2D_PREFETCH", form)
        out[form] = p.adjoint(fd, mode=md).cpu().numpy()
    assert np.array_equal(out["0"], out["1"])
    ref = NF.adjoint_nfft(x, f * w if mode == "dcf" else f, M, sigma, m)
    assert rel(out["1"], ref) < (1e-5 if prec == "fp32" else 1e-12)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("gen", ["random", "clustered"])
def test_spread3d_prefetch_forms_equal(prec, gen, monkeypatch):
    """The d = 3 spread with and without the next points' data prefetched makes the same sums
    in the same order (bit for bit), within the bounds of the oracle's Algorithm 2.4."""
    L, torch = lib_or_skip()
    M, sigma, m = 16, 2.0, 4
    x = points(3, 3000, gen, 31)
    f = inputs.samples_complex(len(x), 32)
    w = inputs.rng(33).uniform(0.5, 1.5, len(x)) / len(x)
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    p = L.Plan(x, M, sigma, m, prec)
    p.set_weights(w.astype(np.complex128))
    fd = to_dev(torch, f, cdt)
    out = {}
    for form in ("0", "1"):
        monkeypatch.setenv("INFFT_SPREAD3D_PREFETCH", form)
        out[form] = p.adjoint(fd, mode=L.MODE_DCF).cpu().numpy()
    assert np.array_equal(out["0"], out["1"])
    ref = NF.adjoint_nfft(x, f * w, M, sigma, m)
    assert rel(out["1"], ref) < (1e-5 if prec == "fp32" else 1e-12)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", ["plain", "dcf", "bopt"])
@pytest.mark.parametrize("M,tile", [(8, 0), (32, 0), (64, 0), (256, 0), (64, 8)])
def test_merge_on_load_equals_merge_kernel(prec, mode, M, tile, monkeypatch):
    """The first FFT pass summing the padded tiles as it loads (Algorithm 2.4 steps 2-3 without
    the grid in between) gives bitwise the result of the halo-merge kernel followed by the
    pass, alone and in a batch of grid sizes; both follow the oracle's Algorithm 2.4 / 4.4.
    M = 8 has one tile (every neighbour wraps onto it), M = 64 with tiles of 8 blocks of 32
    lines spanning four tile rows."""
    L, torch = lib_or_skip()
    if mode == "bopt" and M > 64:
        pytest.skip("B_opt at this size is covered by the headline-size tests")
    N = 3 * M * M
    x = inputs.random_points(N, 2, 800 + M)
    f = inputs.samples_complex(N, 801 + M)
    w = inputs.rng(802 + M).uniform(0.5, 1.5, N) / N
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    tune = {"tile": tile} if tile else None
    p = L.Plan(x, M, 2.0, 4 if mode != "bopt" else 3, prec, tune=tune)
    m = 4 if mode != "bopt" else 3
    md = {"plain": L.MODE_PLAIN, "dcf": L.MODE_DCF, "bopt": L.MODE_BOPT}[mode]
    if mode == "dcf":
        p.set_weights(w.astype(np.complex128))
    if mode == "bopt":
        p.optimize_B()
    fd = to_dev(torch, f, cd)
    q = L.Plan(inputs.random_points(2000, 2, 803), 16, 2.0, m, prec, tune=tune)
    if mode == "dcf":
        q.set_weights(np.full(2000, 1 / 2000, dtype=np.complex128))
    if mode == "bopt":
        q.optimize_B()
    g = to_dev(torch, inputs.samples_complex(2000, 804), cd)
    out, bat = {}, {}
    for form in ("0", "1"):
        monkeypatch.setenv("INFFT_FFT_MERGE", form)
        out[form] = p.adjoint(fd, mode=md).cpu().numpy().ravel()
        h1 = torch.empty((16, 16), dtype=cd, device="cuda")
        h2 = torch.empty((M, M), dtype=cd, device="cuda")
        L.adjoint_batched([q, p], [g, fd], [h1, h2], md)
        bat[form] = h2.cpu().numpy().ravel()
    assert np.array_equal(out["0"], out["1"])
    assert np.array_equal(bat["1"], out["1"])
    assert np.array_equal(bat["0"], bat["1"])
    if mode == "bopt":
        ref = BO.reconstruct(x, f, p.get_bopt(), M, 2.0, m, "kb", BO.PATTERN_2M2)
    else:
        ref = NF.adjoint_nfft(x, f * w if mode == "dcf" else f, M, 2.0, m)
    assert rel(out["1"], ref) < (1e-5 if prec == "fp32" else 1e-12)


@pytest.mark.parametrize("m", [2, 3, 5])
@pytest.mark.parametrize("gen", ["random", "clustered"])
def test_fp32_d2_other_m_match_oracle_algorithm(m, gen):
    """Float32 d = 2 spreading at m = 2, 3 (two points per warp) and m = 5 (one point per warp)
    follows the oracle's Algorithm 2.4 to float32 rounding, on random points and on clustered
    ones (long runs of equal base row, odd run lengths)."""
    L, torch = lib_or_skip()
    M, sigma = 32, 2.0
    x = points(2, 3001, gen, 41)
    f = inputs.samples_complex(len(x), 42)
    p = L.Plan(x, M, sigma, m, "fp32")
    h = p.adjoint(to_dev(torch, f, torch.complex64)).cpu().numpy()
    assert rel(h, NF.adjoint_nfft(x, f, M, sigma, m)) < 1e-5


@pytest.mark.parametrize("N", [1, 2, 3, 31, 32, 33, 65])
def test_fp32_d2_tiny_point_counts(N):
    """One work item of one to 65 points (a lone point leaves the second half-warp idle;
    33 and 65 points cross the 32-point staging and prefetch chunks by one) gives the
    oracle's Algorithm 2.4 to float32 rounding.  M = 8 makes the oversampled grid a single
    16 x 16 tile, so all points form one item."""
    L, torch = lib_or_skip()
    M, sigma, m = 8, 2.0, 3
    x = inputs.random_points(N, 2, 43 + N)
    f = inputs.samples_complex(N, 44 + N)
    p = L.Plan(x, M, sigma, m, "fp32")
    assert p.work_items == 1
    h = p.adjoint(to_dev(torch, f, torch.complex64)).cpu().numpy()
    assert rel(h, NF.adjoint_nfft(x, f, M, sigma, m)) < 1e-5


@pytest.mark.parametrize("M,prec,mode", [
    (32, "fp32", "plain"),     # Ms = 64: one CTA per job
    (64, "fp32", "dcf"),       # Ms = 128: clusters of 2
    (128, "fp32", "plain"),    # Ms = 256: clusters of 8
    (256, "fp32", "dcf"),      # Ms = 512: clusters of 16
    (128, "fp64", "plain"),    # float64 Ms = 256: clusters of 8
    (256, "fp64", "plain"),    # float64 Ms = 512: the two-kernel form
    (32, "fp32", "bopt"),      # B_opt tiles (edge T + 2m + 1)
])
def test_fused_merge_fft_matches_two_kernel_form(monkeypatch, M, prec, mode):
    """The cluster kernel that fuses the halo merge with both FFT passes (Algorithm 2.4
    steps 2-3) gives the two-kernel form's result to rounding (the cells' contributions
    are summed in another fixed order), the oracle's Algorithm 2.4 / 4.4, and the same
    result in a batch as alone."""
    L, torch = lib_or_skip()
    from oracle import bopt as BO
    N = 3 * M * M if mode != "bopt" else 2 * M * M
    x = inputs.random_points(N, 2, 500 + M)
    f = inputs.samples_complex(N, 501 + M)
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    m = 4 if mode != "bopt" else 3
    p = L.Plan(x, M, 2.0, m, prec)
    md, c = L.MODE_PLAIN, f
    if mode == "dcf":
        w = inputs.coeffs_complex((N,), 7) / N
        p.set_weights(w)
        md, c = L.MODE_DCF, w * f
    coef = None
    if mode == "bopt":
        p.optimize_B()
        coef = p.get_bopt()
        md = L.MODE_BOPT
    fd = to_dev(torch, f, cd)
    out = {}
    for form in ("0", "1"):
        monkeypatch.setenv("INFFT_FUSED_MERGE_FFT", form)
        out[form] = p.adjoint(fd, mode=md).cpu().numpy().ravel()
    tol = 1e-6 if prec == "fp32" else 1e-14
    assert rel(out["1"], out["0"]) < tol
    if mode == "bopt":
        ref = BO.reconstruct(x, f, coef, M, 2.0, m, "kb", BO.PATTERN_2M2)
    else:
        ref = NF.adjoint_nfft(x, c, M, 2.0, m)
    assert rel(out["1"], ref) < (1e-5 if prec == "fp32" else 1e-12)
    # alone and in a batch with another set: bit for bit
    monkeypatch.setenv("INFFT_FUSED_MERGE_FFT", "1")
    q = L.Plan(inputs.random_points(5000, 2, 9), M, 2.0, m, prec)
    if mode == "dcf":
        q.set_weights(np.ones(5000) / 5000)
    if mode == "bopt":
        q.optimize_B()
    g = to_dev(torch, inputs.samples_complex(5000, 10), cd)
    h1 = torch.empty((M, M), dtype=cd, device="cuda")
    h2 = torch.empty((M, M), dtype=cd, device="cuda")
    L.adjoint_batched([q, p], [g, fd], [h1, h2], md)
    assert np.array_equal(h2.cpu().numpy().ravel(), out["1"])


@pytest.mark.parametrize("tune", [
    {"tile": 8}, {"item_cap": 64}, {"item_cap": 1024}, {"prefetch": 1}, {"prefetch": 2},
    {"fused_fft": 1}, {"fused_fft": 2}, {"branches": 1}, {"branches": 6},
    {"tile": 8, "item_cap": 100, "prefetch": 2, "fused_fft": 1, "branches": 2},
])
def test_tuned_plans_give_the_same_reconstruction(tune):
    """Kernel choices (infft_tune_t) change speed only: a batch of DCF reconstructions with
    them equals the default to float32 rounding and the oracle's Algorithm 2.4."""
    L, torch = lib_or_skip()
    sets = [(M, inputs.random_points(3 * M * M, 2, 700 + M)) for M in (32, 64, 128)]
    outs = {}
    for key, tn in (("default", None), ("tuned", tune)):
        plans, fs, hs = [], [], []
        for i, (M, x) in enumerate(sets):
            p = L.Plan(x, M, 2.0, 4, "fp32", tune=tn)
            p.set_weights(np.full(x.shape[0], 1.0 / x.shape[0]))
            plans.append(p)
            fs.append(to_dev(torch, inputs.samples_complex(x.shape[0], 710 + i), torch.complex64))
            hs.append(torch.empty((M, M), dtype=torch.complex64, device="cuda"))
        L.adjoint_batched(plans, fs, hs, L.MODE_DCF)
        outs[key] = [h.cpu().numpy().ravel() for h in hs]
    for i, (M, x) in enumerate(sets):
        assert rel(outs["tuned"][i], outs["default"][i]) < 1e-6
        f = inputs.samples_complex(x.shape[0], 710 + i).astype(np.complex64).astype(np.complex128)
        assert rel(outs["tuned"][i], NF.adjoint_nfft(x, f / x.shape[0], M, 2.0, 4)) < 1e-5


@pytest.mark.parametrize("prec,m", [("fp32", 5), ("fp32", 7), ("fp64", 6)])
def test_small_tile_wide_window_d2(prec, m):
    """A tile of 8 with 2m > 8 puts some grid cells in three padded tiles along an axis; the
    reconstruction still follows the oracle's Algorithm 2.4 (the two-source halo merge is not
    used for it)."""
    L, torch = lib_or_skip()
    M = 32
    x = points(2, 3001, "random", 61)
    f = inputs.samples_complex(len(x), 62)
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    p = L.Plan(x, M, 2.0, m, prec, tune={"tile": 8})
    h = p.adjoint(to_dev(torch, f, cdt)).cpu().numpy()
    assert rel(h, NF.adjoint_nfft(x, f, M, 2.0, m)) < (1e-5 if prec == "fp32" else 1e-12)


def test_small_tile_bopt_d2():
    """B_opt's padded tiles hold one more slot per axis (2m + 2): with a tile of 8 at m = 4 some
    cells lie in three tiles along an axis.  Algorithm 4.4 still matches the oracle's with the
    same B_opt."""
    L, torch = lib_or_skip()
    M, m = 16, 4
    x = points(2, 1500, "random", 63)
    f = inputs.samples_complex(len(x), 64)
    p = L.Plan(x, M, 2.0, m, "fp64", tune={"tile": 8})
    p.optimize_B()
    coef = p.get_bopt()
    h = p.adjoint(to_dev(torch, f, torch.complex128), mode=L.MODE_BOPT).cpu().numpy().ravel()
    ref = BO.reconstruct(x, f, coef, M, 2.0, m, "kb", BO.PATTERN_2M2)
    assert rel(h, ref) < 1e-12


def test_invalid_tuning_is_rejected():
    L, torch = lib_or_skip()
    x = inputs.random_points(100, 2, 1)
    for tn in ({"tile": 12}, {"tile": 4}, {"branches": 9}, {"prefetch": 3}, {"item_cap": -1}):
        with pytest.raises(L.InfftError):
            L.Plan(x, 16, 2.0, 4, "fp32", tune=tn)
