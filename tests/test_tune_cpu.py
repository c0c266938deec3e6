"""The autotuner's host logic (no GPU): workload signatures and the JSON cache."""
import json

import numpy as np

import inputs
from paper_2302_00414_gb300 import tune as TU


def test_signature_depends_on_the_workload_only():
    a = [(32, inputs.random_points(5000, 2, 1)), (64, inputs.random_points(20000, 2, 2))]
    b = [(64, inputs.random_points(20000, 2, 3)), (32, inputs.random_points(5000, 2, 4))]
    assert TU.signature(a, 4, "fp32", 1) == TU.signature(b, 4, "fp32", 1)
    assert TU.signature(a, 4, "fp32", 1) != TU.signature(a, 6, "fp32", 1)
    assert TU.signature(a, 4, "fp32", 1) != TU.signature(a, 4, "fp64", 1)
    assert "Ms64-128" in TU.signature(a, 4, "fp32", 1)
    assert TU.A_ms(64, 2.0) == 128 and TU.A_ms(63, 1.0) == 64


def test_cache_round_trip_and_cached_choice(tmp_path):
    path = str(tmp_path / "tuning.json")
    sets = [(16, inputs.random_points(1000, 2, 5))]
    key = TU.signature(sets, 4, "fp32", 1)
    TU.save_cache({key: {"tune": {"branches": 2}, "default_ms": 1.0, "tuned_ms": 0.8}}, path)
    assert json.load(open(path))[key]["tune"] == {"branches": 2}
    got = TU.tuned_choice(None, None, sets, None, 4, "fp32", 1, cache_path=path)
    assert got["source"] == "cache" and got["tune"] == {"branches": 2} and got["key"] == key


def test_candidate_validity():
    assert TU._valid({"tile": 16}, 2, 4)
    assert not TU._valid({"tile": 32}, 2, 4)      # T + 2m + 1 > 32: no register-row spread
    assert not TU._valid({"tile": 4}, 2, 4)       # T <= m
    assert TU._valid({"tile": 8}, 3, 4) and not TU._valid({"tile": 16}, 3, 4)
    assert TU._valid({}, 2, 4) and np.isfinite(1.0)
