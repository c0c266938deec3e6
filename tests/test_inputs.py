"""Seeded generators: shapes, ranges and determinism."""
import numpy as np

import inputs


def test_shapes_and_determinism():
    assert inputs.jittered_1d(256, 0).shape == (256, 1)
    assert np.array_equal(inputs.random_points(100, 2, 3), inputs.random_points(100, 2, 3))
    assert not np.array_equal(inputs.random_points(100, 2, 3), inputs.random_points(100, 2, 4))
    p = inputs.polar(512, 256)
    assert p.shape == (131072, 2)
    # 512 copies of the origin (radius index 0 for every angle)
    assert np.sum(np.all(p == 0, axis=1)) == 512
    s = inputs.spiral_stack(4, 1024, 8)
    assert s.shape == (4096, 3) and s[:, 1:].max() < 0.5 and np.unique(s[:, 0]).size == 4
    assert inputs.linogram(8, 16).shape == (128, 2)
    mp = inputs.modified_polar(8, 16)
    assert np.all((mp >= -0.5) & (mp < 0.5))
    assert inputs.golden_polar(8, 10).shape == (80, 2)


def test_ranges():
    x = inputs.jittered_1d(256, 0)
    assert np.all(np.abs(x[:, 0] - (-0.5 + np.arange(256) / 256)) <= 0.25 / 256)
    r = inputs.random_points(1000, 3, 1)
    assert np.all((r >= -0.5) & (r < 0.5))
    c = inputs.coeffs_complex((50,), 2)
    assert np.all(np.abs(c.real) <= 1) and np.all(np.abs(c.imag) <= 1)
    q = inputs.coeffs_real((50,), 2)
    assert np.all((q.real >= 1) & (q.real <= 10)) and np.all(q.imag == 0)


def test_batch_sets():
    sets = inputs.batch_sets(8, 5)
    assert len(sets) == 8
    for M, x in sets:
        assert M in (32, 64, 128, 256)
        assert 4 * M * M <= x.shape[0] <= 6 * M * M and x.shape[1] == 2
