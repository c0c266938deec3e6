"""Saving and restoring a plan's precompute, so that a cache of point sets survives a restart.

The weights of Algorithm 3.6 and the optimised B of Algorithm 4.3 cost far more than a
reconstruction (seconds to hours in the paper's Table 5.1).  A file holds the plan's
parameters, a SHA-256 digest of the points, a format version and the float64 weights and
B_opt coefficients; restoring rebuilds the plan from the same points (binning is cheap) and
loads the precompute with infft_set_weights / infft_set_bopt.
"""
from __future__ import annotations

import hashlib

import numpy as np

from . import api

FORMAT = 1


def points_digest(x: np.ndarray) -> str:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    h = hashlib.sha256()
    h.update(str(x.shape).encode())
    h.update(x.tobytes())
    return h.hexdigest()


def save_precompute(plan: "api.Plan", x: np.ndarray, path: str) -> None:
    """Write plan parameters, the points' digest and whatever precompute the plan holds."""
    arrays = {"format": np.array(FORMAT), "d": np.array(plan.d), "M": np.array(plan.M),
              "N": np.array(plan.N), "m": np.array(plan.m), "sigma": np.array(plan.sigma),
              "precision": np.array(plan.precision), "window": np.array(plan.window),
              "digest": np.array(points_digest(x))}
    if plan.has_weights:
        arrays["weights"] = plan.get_weights()
    if plan.has_bopt:
        arrays["bopt"] = plan.get_bopt()
    with open(path, "wb") as fh:
        np.savez(fh, **arrays)


def load_precompute(x: np.ndarray, path: str, stream=None, pooled: bool = False) -> "api.Plan":
    """A plan for x with the saved precompute.  Raises ValueError when the file's format
    or the points do not match."""
    with np.load(path, allow_pickle=False) as z:
        if int(z["format"]) != FORMAT:
            raise ValueError(f"precompute format {int(z['format'])}, expected {FORMAT}")
        if str(z["digest"]) != points_digest(x):
            raise ValueError("the points differ from those the precompute was made for")
        plan = api.Plan(x, int(z["M"]), float(z["sigma"]), int(z["m"]), str(z["precision"]),
                        window=str(z["window"]), stream=stream, pooled=pooled)
        if "weights" in z:
            plan.set_weights(np.ascontiguousarray(z["weights"]), stream=stream)
        if "bopt" in z:
            plan.set_bopt(np.ascontiguousarray(z["bopt"]), stream=stream)
    return plan
