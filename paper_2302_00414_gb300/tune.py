"""Autotuner of the library's kernel choices (infft_tune_t in include/infft.h).

For a workload -- a list of point sets of one dimension, precision and window width that
are reconstructed together as one batched, graph-replayed adjoint -- the tuner times the
batch under candidate choices and keeps the fastest:

  tile       spreading tile edge T (d = 2: 16 or 8; the register-row spread needs
             T + 2m + 1 <= 32, so larger tiles are not candidates)
  item_cap   most points per work item (256, 512, 1024)
  prefetch   the spreads' copy of the next points' data to shared memory (on / off)
  fused_fft  the d = 2 cluster kernel that fuses the halo merge with both FFT passes
  branches   concurrent branches of the batch (1, 2, 3, 4, 6)

The search is coordinate descent from the library's defaults (each field in turn over its
values, the others held at the best so far; two sweeps), timed with CUDA events over graph
replays after warm-up.  Results are cached in a JSON file keyed by the workload's
signature: d, the set of oversampled grid sizes, m, the precision, the mode and the total
point count rounded to a power of two.  The choices change speed only: results differ at
most by the rounding of another summation order.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import api as A

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuning.json")

CANDIDATES_2D = {"item_cap": [256, 512, 1024], "prefetch": [1, 2], "fused_fft": [1, 2],
                 "branches": [1, 2, 3, 4, 6], "tile": [16, 8]}
CANDIDATES_3D = {"item_cap": [256, 512, 1024], "prefetch": [1, 2], "branches": [1, 2, 3, 4, 6]}


def signature(sets, m: int, precision: str, mode: int, sigma: float = 2.0) -> str:
    """Cache key of a workload: sets = [(M, x)], x of shape (N, d)."""
    d = sets[0][1].shape[1]
    ms = sorted({A_ms(M, sigma) for M, _ in sets})
    ntot = sum(x.shape[0] for _, x in sets)
    bucket = 1 << max(0, int(round(math.log2(max(1, ntot)))))
    return f"d{d}_Ms{'-'.join(map(str, ms))}_m{m}_{precision}_mode{mode}_sets{len(sets)}_N{bucket}"


def A_ms(M: int, sigma: float) -> int:
    """M_sigma = 2 ceil(ceil(sigma M) / 2) (Section 2.1)."""
    return 2 * math.ceil(math.ceil(sigma * M) / 2)


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE):
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _valid(tune: dict, d: int, m: int) -> bool:
    t = tune.get("tile", 0)
    if t:
        if t <= m:
            return False
        if d == 2 and t + 2 * m + 1 > 32:
            return False
        if d == 3 and t != 8:
            return False
    return True


def time_batch(L, torch, sets, fs, m: int, precision: str, mode: int, tune, sigma: float = 2.0,
               reps: int = 10, warm: int = 3) -> float:
    """Milliseconds per graph replay of the batched adjoint over `sets` with `tune` (None:
    the library's defaults).  Weights (mode DCF) are 1/N: the choices do not depend on them;
    B_opt (mode BOPT) is not supported here."""
    plans, hs = [], []
    cd = torch.complex64 if precision == "fp32" else torch.complex128
    for (M, x) in sets:
        p = L.Plan(x, M, sigma, m, precision, tune=tune)
        if mode == A.MODE_DCF:
            p.set_weights(np.full(x.shape[0], 1.0 / x.shape[0], dtype=np.complex128))
        plans.append(p)
        hs.append(torch.empty((M,) * x.shape[1], dtype=cd, device=fs[0].device))
    batch = L.Batch(plans, fs, hs, mode)
    for _ in range(warm):
        batch.run()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        batch.run()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    batch.close()
    for p in plans:
        p.close()
    return ms


def tune(L, torch, sets, fs, m: int = 4, precision: str = "fp32", mode: int = A.MODE_DCF, sigma: float = 2.0,
         sweeps: int = 2, budget_s: float = 120.0, log=None):
    """Coordinate descent over the candidate choices; returns (best tune dict, default ms,
    best ms, trace list of (tune, ms))."""
    d = sets[0][1].shape[1]
    cand = CANDIDATES_2D if d == 2 else CANDIDATES_3D
    t0 = time.perf_counter()
    trace = []

    def measure(tn):
        ms = time_batch(L, torch, sets, fs, m, precision, mode, tn or None, sigma)
        trace.append((dict(tn), ms))
        if log:
            log(f"tune {tn} -> {ms:.4f} ms")
        return ms

    default_ms = measure({})
    best, best_ms = {}, default_ms
    for _ in range(sweeps):
        improved = False
        for field, values in cand.items():
            for v in values:
                if time.perf_counter() - t0 > budget_s:
                    break
                tn = dict(best)
                tn[field] = v
                if tn == best or not _valid(tn, d, m):
                    continue
                ms = measure(tn)
                if ms < best_ms * 0.995:   # a change must beat the noise of the timing
                    best, best_ms, improved = tn, ms, True
        if not improved:
            break
    return best, default_ms, best_ms, trace


def tuned_choice(L, torch, sets, fs, m: int = 4, precision: str = "fp32", mode: int = A.MODE_DCF,
                 sigma: float = 2.0, cache_path: str = DEFAULT_CACHE, retune: bool = False, log=None) -> dict:
    """The cached choice for this workload, or a fresh search (then cached).  Returns a dict
    with "tune", "default_ms", "tuned_ms", "source", "key" and "search_s"."""
    key = signature(sets, m, precision, mode, sigma)
    cache = load_cache(cache_path)
    if key in cache and not retune:
        out = dict(cache[key])
        out["source"] = "cache"
        out["key"] = key
        return out
    t0 = time.perf_counter()
    best, dms, bms, trace = tune(L, torch, sets, fs, m, precision, mode, sigma, log=log)
    out = {"tune": best, "default_ms": dms, "tuned_ms": bms, "search_s": time.perf_counter() - t0,
           "tried": len(trace)}
    cache[key] = out
    try:
        save_cache(cache, cache_path)
    except OSError:
        pass
    out = dict(out)
    out["source"] = "search"
    out["key"] = key
    return out
