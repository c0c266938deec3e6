"""Checkpoint and restore of a plan's precompute (weights of Algorithm 3.6, B_opt of
Algorithm 4.3): a restored plan reconstructs bit for bit as the original."""
import numpy as np
import pytest

import inputs
from tests.gpu_util import lib_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_saved_precompute_restores_bitwise(tmp_path, prec):
    L, torch = lib_or_skip()
    from paper_2302_00414_gb300 import store
    x = inputs.random_points(1500, 2, 101)
    p = L.Plan(x, 16, 2.0, 3, prec)
    p.weights(max_iter=50)
    p.optimize_B()
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    f = to_dev(torch, inputs.samples_complex(1500, 102), cd)
    h = to_dev(torch, inputs.coeffs_complex((16, 16), 103), cd)
    ref = [p.adjoint(f, mode=L.MODE_DCF), p.adjoint(f, mode=L.MODE_BOPT), p.inverse_adjoint(h)]
    path = str(tmp_path / "plan.npz")
    store.save_precompute(p, x, path)
    q = store.load_precompute(x, path)
    got = [q.adjoint(f, mode=L.MODE_DCF), q.adjoint(f, mode=L.MODE_BOPT), q.inverse_adjoint(h)]
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    assert np.array_equal(q.get_bopt(), p.get_bopt())
    with pytest.raises(ValueError):
        store.load_precompute(x + 1e-9, path)        # other points
