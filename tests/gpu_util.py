"""Helpers for the GPU tests: build/load the library and move arrays to the device."""
import numpy as np
import pytest


def lib_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_00414_gb300 import build as B
    B.build()
    import paper_2302_00414_gb300 as L
    L.load()
    return L, torch


def to_dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
