#!/usr/bin/env python
"""Benchmark of the batched density-compensated iNFFT reconstruction on one GB300.

Workload (the batched two-dimensional configuration): 64 independent point sets,
M_i drawn from {32, 64, 128, 256}, N_i = floor(U(4, 6) M_i^2) i.i.d. uniform points
in [-1/2, 1/2)^2, complex64 samples, Kaiser-Bessel window m = 4, sigma = 2.  Each
set has weights from the library's float64 CG (Algorithm 3.6, capped iterations:
throughput does not depend on weight quality), and one step reconstructs all 64
sets at once, h_i = D^* F^* B^* W_i f_i (Algorithm 3.7), by replaying one CUDA
graph of the batched kernels.

Reported (one JSON line on rank 0):
  value            reconstructions per second over the timed steps (all ranks)
  plain            the same reconstructions issued one at a time, synchronously
  e2e              the same metric through the C ABI with pinned host buffers
                   (host->device copy of f and device->host copy of fhat inside)
  roofline         the spreading kernel's algorithmic bytes / its event-timed
                   duration against the measured HBM copy bandwidth
  rel_err_vs_fp64  max relative l2 error of sampled coefficients against the FP64
                   oracle's exact sums with the same weights
  cpu_baseline     the oracle's exact sums timed on a bounded sample on the host
--impl reference times the FP64 oracle alone (the reference arm of this build).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "iNFFT recon/s & spread GB/s (d=2,M=256) vs plain; p50/p99 ms; rel err vs FP64"
WORKLOAD = ("batched d=2: 64 random point sets, M_i in {32,64,128,256}, N_i=U(4,6)*M_i^2, "
            "DCF reconstruction (Algorithm 3.7), KB m=4, sigma=2, complex64")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sets", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cg-iters", type=int, default=300,
                    help="C3: CG iterations of the weights (Algorithm 3.6); the throughput does not depend on them")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bopt", action="store_true", help="C3: skip the B_opt leg (Algorithms 4.3 / 4.4)")
    ap.add_argument("--no-tune", action="store_true", help="C3: the library's default kernel choices")
    ap.add_argument("--retune", action="store_true", help="C3: search the kernel choices even if cached")
    ap.add_argument("--t51-max", type=int, default=1024, help="T51: largest M of the linogram sweep")
    ap.add_argument("--t51-bopt-max", type=int, default=32, help="T51: largest M with B_opt (Algorithm 4.3)")
    ap.add_argument("--config", default="C3", choices=["C1", "C2", "C3", "C4", "C5", "T51"],
                    help="C3 (default): the batched d=2 workload; C1/C2/C4: single-set workloads; "
                         "C5: Poisson-arrival serving; T51: the linogram sweep in the shape of Table 5.1")
    ap.add_argument("--rate", type=float, default=500.0, help="C5: mean arrival rate (requests/s)")
    ap.add_argument("--requests", type=int, default=20000, help="C5: number of requests")
    ap.add_argument("--new-frac", type=float, default=0.2, help="C5: fraction of requests on new point sets")
    ap.add_argument("--builders", type=int, default=3, help="C5: threads building new point sets")
    ap.add_argument("--bopt-on-admit", action="store_true",
                    help="C5: also optimise B (Algorithm 4.3) on admit and serve with B_opt (Algorithm 4.4)")
    ap.add_argument("--time-limit", type=float, default=120.0, help="C5: wall-clock cap of the serving run (s)")
    return ap.parse_args()


# --------------------------------------------------------------------------------------
# oracle on the host (cpu_baseline / reference arm)

def _oracle_parity(args):
    """The oracle's exact sums for a parity sample, in blocks of about 16M exponentials so
    that sets of millions of points stay within host memory."""
    x, f, M, ks = args
    from oracle import fourier as FO
    return FO.adjoint_ndft(x, f, M, k_subset=ks, chunk=max(1, min(256, (1 << 24) // max(1, x.shape[0]))))


def _oracle_recon(args):
    """One complete reconstruction by the oracle: its float64 Algorithm 2.4 applied to W f
    (Algorithm 3.7), KB m=4, sigma=2.  Returns the seconds it took in this worker."""
    M, x, seed = args
    import inputs
    from oracle import nfft as NF
    N = x.shape[0]
    c = inputs.samples_complex(N, seed) / N      # W f with w_j = 1/N (any weights cost the same)
    t0 = time.perf_counter()
    NF.adjoint_nfft(x, c, M, 2.0, 4)
    return time.perf_counter() - t0


def oracle_sample(sets, step: int, per_m: int):
    """Complete sets for one oracle step: `per_m` sets of every degree M of the batch,
    taken in turn (step k takes the k-th group), so that the sample keeps the batch's
    even mix of M."""
    by_m = {}
    for i, (M, x) in enumerate(sets):
        by_m.setdefault(M, []).append(i)
    pick = []
    for M in sorted(by_m):
        idx = by_m[M]
        for r in range(per_m):
            pick.append(idx[(step * per_m + r) % len(idx)])
    return pick


def oracle_step(sets, pick, pool):
    """Run the oracle on the picked complete sets in the pool; wall seconds of the step."""
    t0 = time.perf_counter()
    pool.map(_oracle_recon, [(sets[i][0], sets[i][1], 1000 + i) for i in pick], chunksize=1)
    return time.perf_counter() - t0


def oracle_sample_text(sets, pick, cores):
    Ms = sorted({sets[i][0] for i in pick})
    return (f"{len(pick)} complete sets per step ({len(pick) // max(1, len(Ms))} of each M in {Ms}) of the "
            f"64-set batch, the oracle's float64 Algorithm 2.4 applied to W f, {cores} worker processes")


# --------------------------------------------------------------------------------------
# replicas on several ranks (one process per GPU, no data-path collective): the timed
# region of every rank, the maximum over ranks, and the whole-job rate

def reduce_over_ranks(x: float, dist, op: str = "max", device=None) -> float:
    """x reduced over all ranks ("max" or "sum"); x itself on one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_rate(units_per_rank: float, ms_local: float, world: int, dist, device=None):
    """Whole-job rate of weak-scaled replicas: all ranks' units over the slowest rank's time.
    Returns (units per second, the slowest rank's milliseconds)."""
    ms = reduce_over_ranks(ms_local, dist, "max", device)
    return world * units_per_rank / (ms / 1e3), ms


# --------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [s.strip() for s in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profiled(name: str = "k_spread2d_batched_d2_m4.md", kernel: str = None):
    """Figures of the committed ncu summary of the spreading kernel (keys "dram_bytes_per_launch",
    "smem_pipe_frac"), or {} when the kernel sources changed since that capture (hash
    mismatch) or the summary covers another instantiation than `kernel`: a stale capture is not
    reported."""
    import hashlib
    summary = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(summary):
        return {}
    h = hashlib.sha256()
    for f in ("spread2d.cuh", "common.cuh", "jobset.cuh"):
        with open(os.path.join(ROOT, "paper_2302_00414_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    want, out, captured = None, {}, None
    for line in open(summary):
        if line.startswith("source_sha256:"):
            want = line.split(":", 1)[1].strip()
        if line.startswith("kernel:"):
            captured = line.split(":", 1)[1].strip()
        for key in ("dram_bytes_per_launch", "smem_pipe_frac"):
            if line.startswith(key + ":"):
                out[key] = float(line.split(":", 1)[1].strip())
    if kernel is not None and captured != kernel:
        return {}
    return out if want == h.hexdigest()[:16] else {}


# FP32 SIMT peak of the GB300 from unit counts and the clock: 152 SMs x 128 FP32 lanes x
# 2 flops per fused multiply-add x 2.07 GHz (derived, not measured)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------------------

def bench_config(sets, world, **extra):
    """The config object of the batched workload (both arms)."""
    cfg = {"workload": WORKLOAD, "sets": len(sets), "d": 2, "M": sorted({M for M, _ in sets}),
           "N_total": int(sum(x.shape[0] for _, x in sets)), "m": 4, "sigma": 2.0, "mode": "DCF",
           "l2": "no flush: per-step inputs (points, weights, samples, scratch) exceed the 129 MB L2",
           "parallelism": f"replicas x{world}"}
    cfg.update(extra)
    return cfg


def run_reference(args, rank, world):
    """The reference arm: the oracle on the host cores.  Each step reconstructs a stratified
    sample of complete sets of the batch (four of every M) with the oracle's float64
    Algorithm 2.4; the step time is the measured wall time of that sample."""
    import inputs
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    sets = inputs.batch_sets(args.sets, args.seed)
    ctx = mp.get_context("spawn")
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    per_m = 4
    with ctx.Pool(cores) as pool:
        for k in range(args.warmup):
            oracle_step(sets, oracle_sample(sets, k, per_m), pool)
        step_s, n_recon = [], 0
        for k in range(args.steps):
            pick = oracle_sample(sets, args.warmup + k, per_m)
            step_s.append(oracle_step(sets, pick, pool))
            n_recon += len(pick)
    total = sum(step_s)
    value = n_recon / total
    sample = oracle_sample_text(sets, pick, cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "recon/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(sets, world),
            "p50_ms": 1e3 * statistics.median(step_s), "p99_ms": 1e3 * float(np.percentile(step_s, 99)),
            "recon_per_step": n_recon // args.steps,
            "cpu_baseline": {"value": value, "unit": "recon/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "recon/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bopt_leg(L, torch, sets, dev, peak, peak_kind, rank):
    """Algorithm 4.3 (B_opt, float64 least squares, 2m+2 slots, KB window) on 16 complete
    sets of the batch (four of every M), then the reconstruction of Algorithm 4.4 on them as
    one graph replay.  Reports the precompute rate, the reconstruction rate, the event-timed
    B_opt spread and its HBM roofline: the spread streams (2m+2)^2 complex64 coefficients
    per point, N (4d + 8 + 8 P) + 8 G bytes per launch (P = (2m+2)^d)."""
    import inputs
    pick = oracle_sample(sets, 0, 4)
    sub = [sets[i] for i in pick]
    plans, fs, hs, res = [], [], [], []
    t0 = time.perf_counter()
    for k, (M, x) in enumerate(sub):
        p = L.Plan(x, M, 2.0, 4, "fp32")
        res.append(p.optimize_B())
        plans.append(p)
        fs.append(torch.from_numpy(inputs.samples_complex(x.shape[0], 3000 + k).astype(np.complex64)).to(dev))
        hs.append(torch.empty((M, M), dtype=torch.complex64, device=dev))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    batch = L.Batch(plans, fs, hs, L.MODE_BOPT)
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize()
    steps = 20
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        batch.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stage = [L.adjoint_batched_timed(plans, fs, hs, L.MODE_BOPT) for _ in range(5)]
    spread_ms = statistics.median(st["spread"] for st in stage)
    Ntot = sum(x.shape[0] for _, x in sub)
    G = sum(p.Ms ** 2 for p in plans)
    Pt = (2 * 4 + 2) ** 2
    nbytes = Ntot * (4 * 2 + 8 + 8 * Pt) + 8 * G
    achieved = nbytes / (spread_ms / 1e3) / 1e9
    err = None
    if rank == 0:   # one M=64 set against the oracle's Algorithm 4.4 with the library's own B_opt
        from oracle import bopt as BO
        i64 = next(k for k, (M, _) in enumerate(sub) if M == 64)
        M, x = sub[i64]
        ref = BO.reconstruct(x, fs[i64].cpu().numpy().astype(np.complex128), plans[i64].get_bopt(), M, 2.0, 4,
                             "kb", BO.PATTERN_2M2)
        got = hs[i64].cpu().numpy().ravel()
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"sets": len(sub), "M": sorted({M for M, _ in sub}), "N_total": int(Ntot),
            "precompute_s": build_s, "builds_per_s": len(sub) / build_s, "max_col_residual": max(res),
            "recon_per_s": len(sub) / (ms / 1e3), "ms_per_step": ms, "spread_ms": spread_ms,
            "rel_err_vs_fp64_alg44": err,
            "roofline": {"bound": "hbm", "kernel": "k_spread2d (B_opt)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                         "algorithmic_bytes": int(nbytes)}}


def run_ours(args, rank, world, dist):
    import torch

    import inputs
    import paper_2302_00414_gb300 as L
    from paper_2302_00414_gb300 import build as B

    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if dist is not None:
        dist.barrier()
    L.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    # ---- set-up (untimed): plans, weights, buffers -------------------------------------
    sets = inputs.batch_sets(args.sets, args.seed + 7919 * rank)
    fs = [torch.from_numpy(inputs.samples_complex(x.shape[0], 1000 + i).astype(np.complex64)).to(dev)
          for i, (M, x) in enumerate(sets)]
    # kernel choices for this workload: the autotuner's cached result, or a fresh search
    tuning = None
    if not args.no_tune:
        from paper_2302_00414_gb300 import tune as TU
        tuning = TU.tuned_choice(L, torch, sets, fs, 4, "fp32", L.MODE_DCF, retune=args.retune)
    tune_cfg = tuning["tune"] if tuning else None
    t_setup = time.perf_counter()
    plans, hs, wres = [], [], []
    t_plan = t_w = 0.0
    for i, (M, x) in enumerate(sets):
        t0 = time.perf_counter()
        p = L.Plan(x, M, 2.0, 4, "fp32", tune=tune_cfg)
        torch.cuda.synchronize()
        t_plan += time.perf_counter() - t0
        t0 = time.perf_counter()
        info = p.weights(max_iter=args.cg_iters, rel_tol=1e-12)
        t_w += time.perf_counter() - t0
        wres.append(info["residual_inf"])
        plans.append(p)
        hs.append(torch.empty((M, M), dtype=torch.complex64, device=dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    Ntot = sum(x.shape[0] for _, x in sets)
    grid_cells = sum(p.Ms ** 2 for p in plans)
    coeffs = sum(M * M for M, _ in sets)

    # the graph of one step; the kernels recorded into it are the launches per step
    L.launch_count_reset()
    batch = L.Batch(plans, fs, hs, L.MODE_DCF)
    kernels_per_step = L.launch_count()
    for _ in range(max(3, args.warmup)):
        batch.run()
    torch.cuda.synchronize()

    # ---- timed region: K graph replays ---------------------------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        e_all0 = torch.cuda.Event(enable_timing=True)
        e_all1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        e_all0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            batch.run()
            ev[k][1].record(stream)
        e_all1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if dist is not None:
        dist.barrier()
    total_ms = e_all0.elapsed_time(e_all1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    recon_per_s, total_ms = replica_rate(len(plans) * args.steps, total_ms, world, dist, dev)

    # ---- stage times (spread roofline) ---------------------------------------------------
    stage = []
    for _ in range(5):
        stage.append(L.adjoint_batched_timed(plans, fs, hs, L.MODE_DCF))
    spread_ms = statistics.median(s["spread"] for s in stage)
    merge_ms = statistics.median(s["merge"] for s in stage)
    fft_ms = [statistics.median(s["fft"][t] for s in stage) for t in range(2)]
    # algorithmic bytes of the DCF spread: N (4d + 8 + 8) + 8 G  (x, f, w; grid written once)
    spread_bytes = Ntot * (4 * 2 + 8 + 8) + 8 * grid_cells
    # flops of the DCF spread: (2m+1)^2 taps of a real window value times a complex sample
    # (two multiply-adds) per point, and the 2 (2m+1) window values (degree-10 polynomials)
    spread_flops = Ntot * ((2 * 4 + 1) ** 2 * 4 + 2 * (2 * 4 + 1) * 2 * 10)
    peak, peak_kind = measured_peak()
    achieved = spread_bytes / (spread_ms / 1e3) / 1e9
    # the paired register-row spread, with or without the prefetching copies as tuned
    spread_kernel = "k_spread2d<float, 4, 0, %d>" % (0 if (tune_cfg or {}).get("prefetch") == 2 else 1)
    prof = profiled(kernel=spread_kernel)
    # merge and the two FFT passes: bytes of the tensors they read and write (the padded
    # tiles as written by the spread), against their event-timed stage
    tile = ((tune_cfg or {}).get("tile") or 16)
    padded = sum(p.work_items * (tile + 2 * 4) ** 2 * 8 for p in plans)   # P = T + 2m per padded edge
    G = grid_cells
    Kc = coeffs
    Mrow = sum(p.Ms * M for p, (M, _) in zip(plans, sets))
    stage_roof = {}
    if merge_ms < 4e-3:   # back-to-back events around no kernel
        # the first pass merges the padded tiles as it loads its rows: no grid in between
        stages = (("merge+fft_pass1", padded + 8 * Mrow, fft_ms[0]),
                  ("fft_pass2", 8 * Mrow + 8 * Kc, fft_ms[1]))
    else:
        stages = (("merge", padded + 8 * G, merge_ms),
                  ("fft_pass1", 8 * G + 8 * Mrow, fft_ms[0]),
                  ("fft_pass2", 8 * Mrow + 8 * Kc, fft_ms[1]))
    for name, nbytes, ms in stages:
        if ms > 0:
            gbs = nbytes / (ms / 1e3) / 1e9
            stage_roof[name] = {"bytes": int(nbytes), "ms": ms, "achieved": gbs, "frac": gbs / peak}

    # ---- the M = 256 sets alone (the metric's "spread GB/s at d=2, M=256"): their spread and
    # passes event-timed as one batch of those sets, bytes as above
    m256 = None
    try:
        sel = [i for i, (M, _) in enumerate(sets) if M == 256]
        if sel:
            P_ = [plans[i] for i in sel]
            st_ = [L.adjoint_batched_timed(P_, [fs[i] for i in sel], [hs[i] for i in sel], L.MODE_DCF)
                   for _ in range(5)]
            sp_ms = statistics.median(s_["spread"] for s_ in st_)
            N_ = sum(sets[i][1].shape[0] for i in sel)
            G_ = sum(p.Ms ** 2 for p in P_)
            sb = N_ * (4 * 2 + 8 + 8) + 8 * G_
            m256 = {"sets": len(sel), "points": int(N_), "spread_ms": sp_ms, "spread_bytes": int(sb),
                    "spread_GBps": sb / (sp_ms / 1e3) / 1e9, "spread_frac": sb / (sp_ms / 1e3) / 1e9 / peak,
                    "fft_ms": [statistics.median(s_["fft"][t_] for s_ in st_) for t_ in range(2)]}
    except Exception as e:   # a report of the subset only: never fail the line for it
        m256 = f"unavailable: {type(e).__name__}"

    # ---- cuFFT on the same grids, as a cross-check baseline of the FFT stage only: full
    # (unpruned) 2D transforms of all 64 oversampled grids, one batched call per grid size
    cufft_ms = None
    try:
        by_ms = {}
        for p in plans:
            by_ms.setdefault(p.Ms, 0)
            by_ms[p.Ms] += 1
        grids = [torch.randn(n, Ms, Ms, dtype=torch.complex64, device=dev) for Ms, n in by_ms.items()]
        for _ in range(3):
            for g in grids:
                torch.fft.fft2(g)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(10):
            for g in grids:
                torch.fft.fft2(g)
        c1.record(stream)
        torch.cuda.synchronize()
        cufft_ms = c0.elapsed_time(c1) / 10
        del grids
    except Exception as e:   # the cross-check is optional
        cufft_ms = f"unavailable: {type(e).__name__}"

    # ---- the persistent form (one launch per step over all 64 sets; off by default because
    # the staged graph above is faster): a graph of it, replayed and event-timed the same way
    persistent = None
    try:
        os.environ["INFFT_PERSISTENT"] = "1"
        hp = [torch.empty_like(h) for h in hs]
        pb = L.Batch(plans, fs, hp, L.MODE_DCF)
        for _ in range(3):
            pb.run()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            pb.run()
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1) / args.steps
        same = all(torch.equal(a, b) for a, b in zip(hp, hs))
        persistent = {"ms_per_step": pms, "recon_per_s": len(plans) / (pms / 1e3), "bitwise_equal_to_staged": same,
                      "wait_timeouts": L.wait_timeouts(),
                      "what": "one persistent kernel per step (spread, merging pass along x, pass along y as "
                              "work units of one queue), graph-replayed; INFFT_PERSISTENT=1"}
        pb.close()
        del hp
    finally:
        os.environ.pop("INFFT_PERSISTENT", None)

    # ---- plain: one reconstruction at a time -----------------------------------------------
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_rounds = 3
    for _ in range(plain_rounds):
        for p, f, h in zip(plans, fs, hs):
            p.adjoint(f, h, L.MODE_DCF)
            torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_rate = plain_rounds * len(plans) / plain_s

    # ---- end to end through the C ABI with pinned host buffers ---------------------------
    # (the graph of one step over page-locked host buffers: every replay copies the step's
    # samples in and its coefficients out; and the same through the per-call API)
    # the step's samples in one page-locked allocation (each set's vector a slice of it), and
    # the results likewise, as a caller batching its requests would hold them
    nf = [int(f.numel()) for f in fs]
    nh = [int(h.numel()) for h in hs]
    f_all = torch.empty(sum(nf), dtype=torch.complex64).pin_memory()
    h_all = torch.empty(sum(nh), dtype=torch.complex64).pin_memory()
    of, oh = np.cumsum([0] + nf), np.cumsum([0] + nh)
    f_host = [f_all[of[i]:of[i + 1]] for i in range(len(fs))]
    h_host = [h_all[oh[i]:oh[i + 1]].view(hs[i].shape) for i in range(len(hs))]
    for a, f in zip(f_host, fs):
        a.copy_(f.cpu())
    fh_np = [t.numpy() for t in f_host]
    hh_np = [t.numpy() for t in h_host]
    hbatch = L.Batch(plans, fh_np, hh_np, L.MODE_DCF)
    for _ in range(3):
        hbatch.run()
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(max(5, min(args.steps, 50))):
        t0 = time.perf_counter()
        hbatch.run()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_rate = world * len(plans) / statistics.median(e2e_times)
    hbatch.close()
    for _ in range(2):
        L.adjoint_batched(plans, fh_np, hh_np, L.MODE_DCF)
    call_times = []
    for _ in range(max(3, min(args.steps, 10))):
        t0 = time.perf_counter()
        L.adjoint_batched(plans, fh_np, hh_np, L.MODE_DCF)
        call_times.append(time.perf_counter() - t0)
    e2e_call_rate = world * len(plans) / statistics.median(call_times)
    h2d = sum(int(f.numel()) * 8 for f in fs)
    d2h = sum(int(h.numel()) * 8 for h in hs)

    # ---- accuracy against the FP64 oracle (sampled coefficients) -------------------------
    rel_errs, e2s = [], []
    if rank == 0:
        from oracle import fourier as FO
        L.adjoint_batched(plans, fs, hs, L.MODE_DCF)
        torch.cuda.synchronize()
        order = sorted(range(len(sets)), key=lambda i: -sets[i][0])
        pick = order[:2] + order[len(order) // 2:len(order) // 2 + 1] + order[-1:]
        rng = np.random.default_rng(1)
        for i in pick:
            M, x = sets[i]
            w = plans[i].get_weights()
            ks = rng.choice(M * M, size=min(64, M * M), replace=False)
            ref = _oracle_parity((x, w * fs[i].cpu().numpy().astype(np.complex128), M, ks))
            got = hs[i].cpu().numpy().ravel()[ks]
            rel_errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        # e_2 = ||h - fhat|| / ||fhat|| of the reconstruction with the capped CG's weights, for
        # data f = A fhat made by a float64 NFFT with a wide window (m = 10)
        for i in pick:
            M, x = sets[i]
            fh = inputs.coeffs_complex((M, M), 9000 + i)
            pf = L.Plan(x, M, 2.0, 10, "fp64")
            fx = pf.forward(np.ascontiguousarray(fh, dtype=np.complex128))
            pf.close()
            hh = plans[i].adjoint(torch.from_numpy(fx.astype(np.complex64)).to(dev), mode=L.MODE_DCF)
            e2s.append({"M": M, "N": int(x.shape[0]), "e2": float(np.linalg.norm(hh.cpu().numpy().ravel() - fh.ravel()) /
                                                               np.linalg.norm(fh)), "residual_inf": wres[i]})

    # ---- B_opt leg: Algorithm 4.3 on a stratified sample of the sets, then Algorithm 4.4 --
    bopt = None
    if not args.no_bopt:
        bopt = bopt_leg(L, torch, sets, dev, peak, peak_kind, rank)

    # ---- CPU baseline: the oracle on complete sets (one reference step) -------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        os.environ["OPENBLAS_NUM_THREADS"] = "1"
        os.environ["OMP_NUM_THREADS"] = "1"
        pick = oracle_sample(sets, 0, 4)
        with mp.get_context("spawn").Pool(cores) as pool:
            wall = oracle_step(sets, pick, pool)
        cpu = {"value": len(pick) / wall, "unit": "recon/s", "cores": cores, "kind": "oracle",
               "sample": oracle_sample_text(sets, pick, cores), "seconds": wall}

    if rank != 0:
        return
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": recon_per_s, "unit": "recon/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(sets, world),
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "plain": {"value": plain_rate, "unit": "recon/s"}, "vs_plain": recon_per_s / world / plain_rate,
        "rel_err_vs_fp64": max(rel_errs) if rel_errs else None,
        "stage_ms": {"spread": spread_ms, "merge": merge_ms, "fft": fft_ms},
        "roofline": {"bound": "smem", "kernel": spread_kernel, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": int(prof["dram_bytes_per_launch"]) if "dram_bytes_per_launch" in prof else None,
                     "peak_kind": peak_kind, "algorithmic_bytes": int(spread_bytes),
                     "binding": {"resource": "shared-memory data pipe (ncu l1tex data-pipe wavefronts)",
                                 "utilization": prof.get("smem_pipe_frac"),
                                 "source": "profiles/k_spread2d_batched_d2_m4.md"},
                     "flops": {"algorithmic": int(spread_flops), "achieved_tflops": spread_flops / (spread_ms / 1e3) / 1e12,
                               "peak_tflops": FP32_PEAK_TFLOPS,
                               "frac": spread_flops / (spread_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                               "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
                     "note": "achieved/peak/frac: HBM (algorithmic bytes / event-timed spread); the kernel is "
                             "bound on chip by the shared-memory pipe"},
        "stage_roofline": stage_roof,
        "persistent": persistent,
        "m256": m256,
        "cufft_crosscheck": {"ms": cufft_ms, "what": "torch.fft.fft2 (cuFFT) of the 64 oversampled grids, "
                             "unpruned, no deconvolution, one batched call per grid size; our two pruned "
                             "passes with deconvolution take stage_ms.fft"},
        "e2e": {"value": e2e_rate, "unit": "recon/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "graph replay over page-locked host buffers (infft_batch_create / infft_batch_run)"},
        "e2e_call": {"value": e2e_call_rate, "unit": "recon/s",
                     "path": "infft_adjoint_batched with page-locked host buffers, one call per step"},
        "gpu_launches": int(kernels_per_step * args.steps),
        "clocks": clocks,
        "precompute": {"setup_s": setup_s, "plan_s": t_plan, "weights_s": t_w, "cg_iters": args.cg_iters,
                       "weights_residual_max": max(wres), "e2_vs_fhat": e2s},
        "cpu_baseline": cpu,
        "bopt": bopt,
        "tuning": tuning,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# single-set workloads (one reconstruction per step)

def config_sets(name):
    """(label, d, M, m list, precision, points, workload text) of the single-set workloads;
    inputs are seeded with 1000 * config index + set index."""
    import inputs
    if name == "C1":
        return ("C1", 1, 64, [6], "fp64", inputs.jittered_1d(256, 1000),
                "d=1, M=64, sigma=2, m=6, N=256 jittered points, FP64 transform and weights")
    if name == "C2":
        return ("C2", 2, 128, [4, 6], "fp32", inputs.polar(512, 256),
                "d=2, M=128, sigma=2, polar grid 512 angles x 256 radii (N=131072), m in {4,6}, FP32 "
                "reconstruction, FP64 weights at degree 256")
    return ("C4", 3, 64, [4], "fp32", inputs.spiral_stack(64, 32768, 64),
            "d=3, M=64, sigma=2 (grid 128^3), stack of 64 spirals x 32768 points (N=2^21), m=4, FP32 "
            "reconstruction, FP64 weights at degree 128")


def run_single(args, rank, world, dist):
    import torch

    import inputs
    import paper_2302_00414_gb300 as L
    from oracle import fourier as FO
    from paper_2302_00414_gb300 import build as B

    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if dist is not None:
        dist.barrier()
    L.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    label, d, M, ms, prec, x, workload = config_sets(args.config)
    N = x.shape[0]
    cidx = int(label[1])
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    cbytes = 16 if prec == "fp64" else 8
    if label == "C1":
        fh_true = inputs.coeffs_complex((M,), 1000 * cidx)
        f_np = FO.ndft(x, fh_true, M)           # f = A fhat by the oracle's exact sums
    else:
        # f = A fhat for random fhat by a float64 NFFT of the library with a wide window
        # (m = 10 for d = 2, 6 for d = 3; error ~1e-14), as the paper makes its data by an
        # NFFT: e_2 = ||h - fhat|| / ||fhat|| then measures the weights and the reconstruction
        fh_true = inputs.coeffs_complex((M,) * d, 1000 * cidx)
        pf = L.Plan(x, M, 2.0, 10 if d == 2 else 6, "fp64")
        f_np = pf.forward(np.ascontiguousarray(fh_true, dtype=np.complex128))
        pf.close()
    cg_iters = {"C1": 500, "C2": 30, "C4": 10}[label]
    per_m = {}
    for m in ms:
        p = L.Plan(x, M, 2.0, m, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = p.weights(max_iter=cg_iters, rel_tol=1e-14 if label == "C1" else 1e-12)
        t_w = time.perf_counter() - t0
        w = p.get_weights()
        f = torch.from_numpy(f_np.astype(np.complex128 if prec == "fp64" else np.complex64)).to(dev)
        h = torch.empty((M,) * d, dtype=cdt, device=dev)
        L.launch_count_reset()
        batch = L.Batch([p], [f], [h], L.MODE_DCF)
        kernels_per_step = L.launch_count()
        for _ in range(max(3, args.warmup)):
            batch.run()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev.index) as clk:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.steps):
                ev[k][0].record(stream)
                batch.run()
                ev[k][1].record(stream)
            e1.record(stream)
            torch.cuda.synchronize()
        total_ms = reduce_over_ranks(e0.elapsed_time(e1), dist, "max", dev)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        stage = [L.adjoint_batched_timed([p], [f], [h], L.MODE_DCF) for _ in range(5)]
        st = {"spread": statistics.median(s_["spread"] for s_ in stage),
              "merge": statistics.median(s_["merge"] for s_ in stage),
              "fft": [statistics.median(s_["fft"][t_] for s_ in stage) for t_ in range(d)]}
        G, K = p.Ms ** d, M ** d
        spread_bytes = N * (4 * d + cbytes + cbytes) + cbytes * G     # x, f, w; grid once
        fft_bytes = cbytes * G + cbytes * K                            # ideal single pass
        gbs = {"spread": spread_bytes / (st["spread"] / 1e3) / 1e9,
               "fft_total": fft_bytes / (sum(st["fft"]) / 1e3) / 1e9}
        # every stage against HBM: the merge reads the padded tiles once (P = T + 2m per edge, the
        # library's default tile edge) and writes the grid; FFT pass t reads Ms^(d-t) M^t and
        # writes Ms^(d-t-1) M^(t+1) elements
        T_def = min(256, p.Ms) if d == 1 else (16 if d == 2 else 8)
        merge_bytes = p.work_items * (T_def + 2 * m) ** d * cbytes + cbytes * G
        stage_roof = {"spread": {"bytes": int(spread_bytes), "ms": st["spread"]}}
        if st["merge"] > 4e-3:
            stage_roof["merge"] = {"bytes": int(merge_bytes), "ms": st["merge"]}
        for t_ in range(d):
            nb = cbytes * (p.Ms ** (d - t_) * M ** t_ + p.Ms ** (d - t_ - 1) * M ** (t_ + 1))
            stage_roof[f"fft_pass{t_ + 1}"] = {"bytes": int(nb), "ms": st["fft"][t_]}
        pk, _ = measured_peak()
        for v_ in stage_roof.values():
            v_["achieved"] = v_["bytes"] / (v_["ms"] / 1e3) / 1e9 if v_["ms"] > 0 else None
            v_["frac"] = v_["achieved"] / pk if v_["achieved"] else None
        # plain and end to end
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            p.adjoint(f, h, L.MODE_DCF)
            torch.cuda.synchronize()
        plain_rate = 10 / (time.perf_counter() - t0)
        f_host = f.cpu().pin_memory()
        h_host = torch.empty(h.shape, dtype=h.dtype).pin_memory()
        fh_np, hh_np = f_host.numpy(), h_host.numpy()
        L.adjoint_batched([p], [fh_np], [hh_np], L.MODE_DCF)
        e2e = []
        for _ in range(10):
            t0 = time.perf_counter()
            L.adjoint_batched([p], [fh_np], [hh_np], L.MODE_DCF)
            e2e.append(time.perf_counter() - t0)
        # parity with the oracle's exact sums (same weights) on sampled coefficients
        L.adjoint_batched([p], [f], [h], L.MODE_DCF)
        torch.cuda.synchronize()
        nk = {"C1": K, "C2": 1024, "C4": 4096}[label]
        ks = np.random.default_rng(1000 * cidx + 2).choice(K, size=min(nk, K), replace=False)
        t0 = time.perf_counter()
        wf = w * f_np
        if len(ks) * N > 10 ** 8:   # large sample: the exact sums on all host cores
            cores = len(os.sched_getaffinity(0))
            with mp.get_context("spawn").Pool(cores) as pool:
                parts = pool.map(_oracle_parity, [(x, wf, M, c) for c in np.array_split(ks, cores) if len(c)])
            ref = np.concatenate(parts)
        else:
            ref = _oracle_parity((x, wf, M, ks))
        oracle_s = time.perf_counter() - t0
        got = h.cpu().numpy().ravel()[ks]
        rec = {"recon_per_s": world * args.steps / (total_ms / 1e3), "ms_per_step": total_ms / args.steps,
               "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
               "plain_recon_per_s": plain_rate, "e2e_recon_per_s": world / statistics.median(e2e),
               "stage_ms": st, "stage_GBps": gbs, "stage_roofline": stage_roof,
               "spread_algorithmic_bytes": int(spread_bytes),
               "rel_err_vs_O1": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
               "O1_sampled_k": int(len(ks)), "O1_seconds": oracle_s,
               "weights": {"seconds": t_w, "cg_iters": info["iters"], "residual_inf": info["residual_inf"]},
               "gpu_launches": int(kernels_per_step * args.steps), "clocks": clk.summary(),
               "h2d_bytes_per_step": N * cbytes, "d2h_bytes_per_step": K * cbytes}
        if fh_true is not None:
            rec["e2_vs_fhat"] = float(np.linalg.norm(h.cpu().numpy().ravel() - fh_true.ravel()) /
                                      np.linalg.norm(fh_true))
        per_m[m] = rec
        batch.close()
        p.close()
    if rank != 0:
        return
    head = per_m[ms[0]]
    peak, peak_kind = measured_peak()
    line = {
        "metric": f"iNFFT recon/s, {label} (single set); rel err vs O1", "value": head["recon_per_s"],
        "unit": "recon/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": workload, "name": label, "d": d, "M": M, "N": int(N), "m": ms, "sigma": 2.0,
                   "mode": "DCF", "l2": "inputs and grids exceed L2" if label == "C4" else
                   "small case: inputs fit in L2 (no flush)", "parallelism": f"replicas x{world}"},
        "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
        "plain": {"value": head["plain_recon_per_s"], "unit": "recon/s"},
        "roofline": {"bound": "hbm", "kernel": "spread", "achieved": head["stage_GBps"]["spread"], "peak": peak,
                     "unit": "GB/s", "frac": head["stage_GBps"]["spread"] / peak, "traffic": None,
                     "peak_kind": peak_kind, "algorithmic_bytes": head["spread_algorithmic_bytes"]},
        "stage_roofline": head["stage_roofline"],
        "e2e": {"value": head["e2e_recon_per_s"], "unit": "recon/s",
                "h2d_bytes_per_step": head["h2d_bytes_per_step"], "d2h_bytes_per_step": head["d2h_bytes_per_step"]},
        "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
        "per_m": {str(k): v for k, v in per_m.items()},
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# Poisson-arrival serving (continuous batching over the C ABI)

SERVE_CLASSES = [(2, 64), (2, 128), (2, 256), (3, 32), (3, 64)]


def serve_point_set(rng):
    """A point set of the serving workload: class (d, M) uniform over SERVE_CLASSES,
    N = floor(|I_2M| U(1, 1.5)), uniform random points, or a polar grid for half of the
    two-dimensional sets.  Returns (d, M, N, make) with make() generating the points
    (deterministic), so that thousands of sets need no host memory until built."""
    import inputs
    d, M = SERVE_CLASSES[int(rng.integers(len(SERVE_CLASSES)))]
    N = int((2 * M) ** d * rng.uniform(1.0, 1.5))
    seed = int(rng.integers(2 ** 31))
    if d == 2 and rng.uniform() < 0.5:
        na = int(np.sqrt(2 * N))
        nr = max(2, N // na)
        return d, M, na * nr, lambda: inputs.polar(na, nr)
    return d, M, N, lambda: inputs.random_points(N, d, seed)


def run_serving(args, rank, world, dist):
    import torch

    import paper_2302_00414_gb300 as L
    from paper_2302_00414_gb300 import build as B
    from paper_2302_00414_gb300.serve import Backend, PointSet, Request, Server, latency_summary, run_poisson

    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if dist is not None:
        dist.barrier()
    L.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(5000 + rank)
    cg_iters = min(args.cg_iters, 10)
    be = Backend(weights_iters=cg_iters, bopt=args.bopt_on_admit)
    budget = int(0.5 * torch.cuda.mem_get_info()[0])
    kept = {}

    def keep(r):   # a few results of small sets for the parity check; the rest is dropped
        d, M, _ = meta[r.key]
        if M <= 64 and len(kept) < 3 and r.key not in kept:
            kept[r.key] = r.rid
            return True
        return False

    server = Server(be, mem_budget=budget, max_batch=32, streams=3, keep_output=keep, builders=args.builders)
    meta = {}
    # one sample buffer per class, long enough for its largest N; a request on a set
    # with N points reads the first N entries
    pool = {c: torch.randn(int((2 * c[1]) ** c[0] * 1.5) + 1, dtype=torch.complex64, device=dev)
            for c in SERVE_CLASSES}
    samples = {}

    def register(key, pin=False):
        d, M, N, make = serve_point_set(rng)
        server.register(PointSet(key, d, M, make, N=N), pin=pin)
        samples[key] = pool[(d, M)][:N]
        meta[key] = (d, M, make)

    # cached plans: two sets per class, precomputed before the timed run and kept
    keys = []
    for c in range(2 * len(SERVE_CLASSES)):
        register(c, pin=True)
        keys.append(c)
    warm = [Request(rid=-1 - k, key=k, f=samples[k]) for k in keys]
    for r in warm:
        server.submit(r)
    server.drain(timeout=600)
    server.completed.clear()
    server.stats.clear()
    server.launch_times.clear()
    be.launch_max.clear()
    be.launch_sum.clear()
    kept.clear()
    be.phase_s.clear()
    n_warm_builds = len(server.build_times)

    # request stream: a fraction on new point sets (precomputed on admit), the rest on
    # the cached sets
    reqs, is_new = [], {}
    next_key = len(keys)
    for i in range(args.requests):
        if rng.uniform() < args.new_frac:
            register(next_key)
            k = next_key
            next_key += 1
            is_new[i] = True
        else:
            k = keys[int(rng.integers(len(keys)))]
            is_new[i] = False
        reqs.append(Request(rid=i, key=k, f=samples[k]))
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        done = run_poisson(server, reqs, args.rate, seed=rank, time_limit=args.time_limit)
        wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    done = list(done)
    server.abort()
    summ = latency_summary(done)
    cached = [r for r in done if not is_new[r.rid]]
    new = [r for r in done if is_new[r.rid]]
    builds = server.build_times[n_warm_builds:]
    by_class = {}
    for key, sec in builds:
        d, M, _ = meta[key]
        by_class.setdefault(f"d{d}M{M}", []).append(sec)
    # parity of a few served results with the oracle's exact sums (same weights)
    rel_errs, e2s = [], []
    if rank == 0:
        from oracle import fourier as FO
        picks = [r for r in done if r.out is not None and r.key in server.plans][:3]
        krng = np.random.default_rng(5)
        for r in picks:
            d, M, make = meta[r.key]
            x = make()
            w = server.plans[r.key].get_weights()
            ks = krng.choice(M ** d, size=64, replace=False)
            ref = _oracle_parity((x, w * r.f.cpu().numpy().astype(np.complex128), M, ks))
            got = r.out.cpu().numpy().ravel()[ks]
            rel_errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    thr = reduce_over_ranks(len(done) / wall, dist, "sum", dev)
    if rank != 0:
        return
    line = {
        "metric": "iNFFT serving: p50/p99 ms, recon/s under Poisson arrivals", "value": thr,
        "unit": "recon/s", "n_gpus": world, "steps": len(done), "warmup": len(warm),
        "ms_per_step": 1e3 * wall / max(1, len(done)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "C5 serving: Poisson arrivals, classes d=2 M in {64,128,256}, d=3 M in {32,64}, "
                               "N = |I_2M| U(1,1.5), random or polar points; new point sets precomputed on "
                               "admit (plan + FP64 weights), cached plans reused",
                   "name": "C5", "rate_per_s": args.rate, "requests": args.requests, "new_frac": args.new_frac,
                   "time_limit_s": args.time_limit, "cg_iters": cg_iters, "max_batch": 32, "streams": 3,
                   "mem_budget_bytes": budget, "parallelism": f"replicas x{world}"},
        "completed": len(done), "submitted_within_limit": sum(1 for r in reqs if r.t_arrive > 0),
        "wall_s": wall, "p50_ms": summ.get("p50_ms"), "p99_ms": summ.get("p99_ms"),
        "latency_all": summ, "latency_cached": latency_summary(cached), "latency_new_set": latency_summary(new),
        "precompute_s_by_class": {k: {"n": len(v), "mean": float(np.mean(v)), "max": float(np.max(v))}
                                  for k, v in by_class.items()},
        "server_stats": dict(server.stats), "rel_err_vs_O1": max(rel_errs) if rel_errs else None,
        "launch_host_ms": ({"p50": 1e3 * float(np.percentile(server.launch_times, 50)),
                            "p99": 1e3 * float(np.percentile(server.launch_times, 99)),
                            "max": 1e3 * float(np.max(server.launch_times))} if server.launch_times else None),
        "build_phase_s": dict(be.phase_s),
        "launch_phase_max_ms": {k: 1e3 * v for k, v in be.launch_max.items()},
        "launch_phase_sum_s": dict(be.launch_sum),
        "e2e": {"value": thr, "unit": "recon/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "samples resident on the device; latency measured from arrival to completion event"},
        "gpu_launches": None, "clocks": clk.summary(), "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# linogram sweep in the shape of Table 5.1 (random coefficients in place of the phantom)

def _timed_recon(L, torch, p, f, h, mode, steps):
    b = L.Batch([p], [f], [h], mode)
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        b.run()
    e1.record(st)
    torch.cuda.synchronize()
    b.close()
    return e0.elapsed_time(e1) / steps


def run_table51(args, rank, world, dist):
    """M = 2^c, linogram grid R = 2M, T = 2R (N = 8 M^2 > |I_2M|), f = A fhat for random fhat:
    relative error e_2 = ||h - fhat|| / ||fhat|| (eq. relative_errors), precompute and
    reconstruction times of Algorithm 3.7 (weights of Algorithm 3.6, here FP64 with m = 8,
    sigma = 2, and the FP32 fast path with m = 4) and of Algorithm 4.4 (B_opt of Algorithm 4.3,
    FP64, sigma = 1, m = 4 as the paper states, with the Dirichlet window, the optimal one of
    Theorem 4.5; the Kaiser-Bessel window gave e_2 = 1.5e-4 at M = 16).  From M = 64 on, the
    columns at the grid's centre (all radii meet there) exceed what one column solve holds in
    shared memory, so B_opt stops at --t51-bopt-max."""
    import torch

    import inputs
    import paper_2302_00414_gb300 as L
    from oracle import fourier as FO
    from paper_2302_00414_gb300 import build as B
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if dist is not None:
        dist.barrier()
    L.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    rows = []
    M = 16
    t_all = time.perf_counter()
    while M <= args.t51_max:
        x = inputs.linogram(2 * M, 4 * M)
        N = x.shape[0]
        fh = inputs.coeffs_complex((M, M), 5100 + M)
        if N * M * M <= 2e9:   # the oracle's exact sums
            f = FO.ndft(x, fh, M)
            f_src = "exact sums (oracle)"
        else:                   # as the paper: an NFFT of fhat (the library's FP64 NFFT, m = 10)
            q = L.Plan(x, M, 2.0, 10, "fp64")
            f = q.forward(torch.from_numpy(fh).to(dev)).cpu().numpy()
            q.close()
            f_src = "FP64 NFFT, m=10"
        row = {"M": M, "N": int(N), "f": f_src}
        fd = torch.from_numpy(f).to(dev)
        # Algorithm 3.7, FP64
        p = L.Plan(x, M, 2.0, 8, "fp64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = p.weights(max_iter=500, rel_tol=1e-14)
        row["dcf_fp64_precompute_s"] = time.perf_counter() - t0
        row["dcf_fp64_cg_iters"] = info["iters"]
        row["dcf_weight_residual"] = info["residual_inf"]
        h = torch.empty((M, M), dtype=torch.complex128, device=dev)
        row["dcf_fp64_recon_ms"] = _timed_recon(L, torch, p, fd, h, L.MODE_DCF, 10)
        row["dcf_fp64_e2"] = float(np.linalg.norm(h.cpu().numpy() - fh) / np.linalg.norm(fh))
        w = p.get_weights()
        p.close()
        # Algorithm 3.7, FP32 fast path with the same weights
        p = L.Plan(x, M, 2.0, 4, "fp32")
        p.set_weights(w)
        f32 = fd.to(torch.complex64)
        h32 = torch.empty((M, M), dtype=torch.complex64, device=dev)
        row["dcf_fp32_recon_ms"] = _timed_recon(L, torch, p, f32, h32, L.MODE_DCF, 20)
        row["dcf_fp32_e2"] = float(np.linalg.norm(h32.cpu().numpy() - fh) / np.linalg.norm(fh))
        p.close()
        # Algorithm 4.4
        if M <= args.t51_bopt_max:
            p = L.Plan(x, M, 1.0, 4, "fp64", window="dirichlet")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.optimize_B()
            row["bopt_precompute_s"] = time.perf_counter() - t0
            hb = torch.empty((M, M), dtype=torch.complex128, device=dev)
            row["bopt_recon_ms"] = _timed_recon(L, torch, p, fd, hb, L.MODE_BOPT, 10)
            row["bopt_e2"] = float(np.linalg.norm(hb.cpu().numpy() - fh) / np.linalg.norm(fh))
            p.close()
        rows.append(row)
        print(json.dumps({"t51_row": row}), file=sys.stderr, flush=True)
        M *= 2
    if rank != 0:
        return
    head = rows[-1]
    line = {
        "metric": "iNFFT recon time and e_2 on linogram grids (Table 5.1 shapes)",
        "value": 1e3 / head["dcf_fp32_recon_ms"], "unit": "recon/s", "n_gpus": world, "steps": 10,
        "warmup": 3, "ms_per_step": head["dcf_fp32_recon_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "linogram R=2M, T=2R, N=8M^2, random fhat in place of the phantom; "
                               "value: FP32 DCF reconstruction at the largest M", "name": "T51",
                   "M": [r["M"] for r in rows]},
        "rows": rows, "wall_s": time.perf_counter() - t_all,
        "roofline": None, "e2e": None, "gpu_launches": None, "clocks": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist_mod
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.config in ("C1", "C2", "C4"):
            run_single(args, rank, world, dist)
        elif args.config == "C5":
            run_serving(args, rank, world, dist)
        elif args.config == "T51":
            run_table51(args, rank, world, dist)
        else:
            run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
