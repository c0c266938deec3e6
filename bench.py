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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sets", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cg-iters", type=int, default=25)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# --------------------------------------------------------------------------------------
# oracle on the host (cpu_baseline / reference arm)

def _oracle_chunk(args):
    x, f, M, ks = args
    from oracle import fourier as FO
    return FO.adjoint_ndft(x, f, M, k_subset=ks)


def oracle_cost(x, f, M, seconds, pool, cores, seed=0):
    """Time the oracle's exact adjoint sums (eq. nfft*) for a bounded random subset of
    I_M: one calibration chunk, then one chunk sized to fill about `seconds`.  Returns
    (seconds per point and coefficient, description of the sample)."""
    K = M * M
    N = x.shape[0]
    rng = np.random.default_rng(seed)

    def run(n):
        ks = rng.choice(K, size=min(n, K), replace=False)
        chunks = [(x, f, M, c) for c in np.array_split(ks, cores) if len(c)]
        t0 = time.perf_counter()
        pool.map(_oracle_chunk, chunks)
        return time.perf_counter() - t0, len(ks)

    t1, n1 = run(cores)
    n2 = int(max(0.0, seconds - t1) / (t1 / n1))
    t2, n2 = run(n2) if n2 > 0 else (0.0, 0)
    cost = (t1 + t2) / ((n1 + n2) * N)
    return cost, f"{n1 + n2} of {K} coefficients of one M={M}, N={N} set (exact sums), extrapolated by N*M^2"


def batch_rate_from_cost(cost, sets):
    """Reconstructions per second of the whole batch at `cost` seconds per point-coefficient."""
    return len(sets) / sum(cost * x.shape[0] * M * M for M, x in sets)


# --------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")
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


def profiled_traffic():
    """DRAM bytes per launch of the spreading kernel from the committed ncu summary, or
    None when the kernel sources changed since that capture (hash mismatch)."""
    import hashlib
    summary = os.path.join(ROOT, "profiles", "k_spread2d_batched_d2_m4.md")
    if not os.path.exists(summary):
        return None
    h = hashlib.sha256()
    for f in ("nfft.cu", "common.cuh", "jobset.cuh"):
        with open(os.path.join(ROOT, "paper_2302_00414_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    want, value = None, None
    for line in open(summary):
        if line.startswith("source_sha256:"):
            want = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            value = int(line.split(":", 1)[1].strip())
    return value if want == h.hexdigest()[:16] else None


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------------------

def run_reference(args, rank, world):
    import inputs
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    sets = inputs.batch_sets(args.sets, args.seed)
    M, x = max(sets, key=lambda s: s[0] * 10 ** 9 + s[1].shape[0])
    f = inputs.samples_complex(x.shape[0], 1)
    ctx = mp.get_context("spawn")
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    per_step = min(10.0, max(0.5, 150.0 / max(1, args.steps + args.warmup)))
    with ctx.Pool(cores) as pool:
        for k in range(args.warmup):
            oracle_cost(x, f, M, per_step / 4, pool, cores, seed=k)
        rates = []
        t0 = time.perf_counter()
        for k in range(args.steps):
            cost, sample = oracle_cost(x, f, M, per_step, pool, cores, seed=100 + k)
            rates.append(batch_rate_from_cost(cost, sets))
        wall = time.perf_counter() - t0
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "recon/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * len(sets) / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; reference = FP64 exact sums (oracle) on the host",
                       "sample_set": {"M": M, "N": int(x.shape[0])},
                       "note": "each step times a bounded sample of one M=256 set and extrapolates the "
                               "whole 64-set batch by N_i*M_i^2"},
            "cpu_baseline": {"value": value, "unit": "recon/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "recon/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


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
    t_setup = time.perf_counter()
    plans, fs, hs, wres = [], [], [], []
    t_plan = t_w = 0.0
    for i, (M, x) in enumerate(sets):
        t0 = time.perf_counter()
        p = L.Plan(x, M, 2.0, 4, "fp32")
        torch.cuda.synchronize()
        t_plan += time.perf_counter() - t0
        t0 = time.perf_counter()
        info = p.weights(max_iter=args.cg_iters, rel_tol=1e-12)
        t_w += time.perf_counter() - t0
        wres.append(info["residual_inf"])
        f = torch.from_numpy(inputs.samples_complex(x.shape[0], 1000 + i).astype(np.complex64)).to(dev)
        plans.append(p)
        fs.append(f)
        hs.append(torch.empty((M, M), dtype=torch.complex64, device=dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    Ntot = sum(x.shape[0] for _, x in sets)
    grid_cells = sum(p.Ms ** 2 for p in plans)
    coeffs = sum(M * M for M, _ in sets)

    # kernels per batched reconstruction
    L.launch_count_reset()
    L.adjoint_batched(plans, fs, hs, L.MODE_DCF)
    torch.cuda.synchronize()
    kernels_per_step = L.launch_count()

    batch = L.Batch(plans, fs, hs, L.MODE_DCF)
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
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    recon_per_s = world * len(plans) * args.steps / (total_ms / 1e3)

    # ---- stage times (spread roofline) ---------------------------------------------------
    stage = []
    for _ in range(5):
        stage.append(L.adjoint_batched_timed(plans, fs, hs, L.MODE_DCF))
    spread_ms = statistics.median(s["spread"] for s in stage)
    merge_ms = statistics.median(s["merge"] for s in stage)
    fft_ms = [statistics.median(s["fft"][t] for s in stage) for t in range(2)]
    # algorithmic bytes of the DCF spread: N (4d + 8 + 8) + 8 G  (x, f, w; grid written once)
    spread_bytes = Ntot * (4 * 2 + 8 + 8) + 8 * grid_cells
    peak, peak_kind = measured_peak()
    achieved = spread_bytes / (spread_ms / 1e3) / 1e9

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
    f_host = [f.cpu().pin_memory() for f in fs]
    h_host = [torch.empty(h.shape, dtype=h.dtype).pin_memory() for h in hs]
    fh_np = [t.numpy() for t in f_host]
    hh_np = [t.numpy() for t in h_host]
    for _ in range(2):
        L.adjoint_batched(plans, fh_np, hh_np, L.MODE_DCF)
    e2e_times = []
    for _ in range(max(3, min(args.steps, 10))):
        t0 = time.perf_counter()
        L.adjoint_batched(plans, fh_np, hh_np, L.MODE_DCF)
        e2e_times.append(time.perf_counter() - t0)
    e2e_rate = world * len(plans) / statistics.median(e2e_times)
    h2d = sum(int(f.numel()) * 8 for f in fs)
    d2h = sum(int(h.numel()) * 8 for h in hs)

    # ---- accuracy against the FP64 oracle (sampled coefficients) -------------------------
    rel_errs = []
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
            ref = FO.adjoint_ndft(x, w * fs[i].cpu().numpy().astype(np.complex128), M, k_subset=ks)
            got = hs[i].cpu().numpy().ravel()[ks]
            rel_errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))

    # ---- CPU baseline: the oracle on a bounded sample --------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        M, x = max(sets, key=lambda s: s[0] * 10 ** 9 + s[1].shape[0])
        f = inputs.samples_complex(x.shape[0], 1)
        os.environ["OPENBLAS_NUM_THREADS"] = "1"
        os.environ["OMP_NUM_THREADS"] = "1"
        with mp.get_context("spawn").Pool(cores) as pool:
            cost, sample = oracle_cost(x, f, M, args.cpu_seconds, pool, cores)
        cpu = {"value": batch_rate_from_cost(cost, sets), "unit": "recon/s", "cores": cores, "kind": "oracle",
               "sample": sample}

    if rank != 0:
        return
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": recon_per_s, "unit": "recon/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sets": len(plans), "d": 2, "M": sorted({M for M, _ in sets}),
                   "N_total": int(Ntot), "m": 4, "sigma": 2.0, "mode": "DCF",
                   "l2": "no flush: per-step inputs (points, weights, samples, scratch) exceed the 129 MB L2",
                   "parallelism": f"replicas x{world}"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "plain": {"value": plain_rate, "unit": "recon/s"}, "vs_plain": recon_per_s / world / plain_rate,
        "rel_err_vs_fp64": max(rel_errs) if rel_errs else None,
        "stage_ms": {"spread": spread_ms, "merge": merge_ms, "fft": fft_ms},
        "roofline": {"bound": "hbm", "kernel": "k_spread2d", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": profiled_traffic(),
                     "peak_kind": peak_kind, "algorithmic_bytes": int(spread_bytes),
                     "note": "issue-bound (ncu: 67% issue active, DRAM 7%), see profiles/"},
        "e2e": {"value": e2e_rate, "unit": "recon/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(kernels_per_step * args.steps),
        "clocks": clocks,
        "precompute": {"setup_s": setup_s, "plan_s": t_plan, "weights_s": t_w, "cg_iters": args.cg_iters,
                       "weights_residual_max": max(wres)},
        "cpu_baseline": cpu,
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
        else:
            run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
