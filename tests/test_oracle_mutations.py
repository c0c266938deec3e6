"""Planted mistakes in the oracle must break a pin.

Each case patches one step of the oracle on the CPU (a sign, a dropped factor,
a swapped size, a transposed operand) and re-runs a pin check, which must
now fail.  This shows that the pins constrain the parts they are meant to.
"""
import numpy as np
import pytest

import inputs
from oracle import fourier as FO
from oracle import nfft as NF
from oracle import weights as WT
from oracle import windows as W


def _nfft_pin():
    x = inputs.random_points(300, 2, 11)
    f = inputs.samples_complex(300, 12)
    ref = FO.adjoint_ndft(x, f, 16)
    err = np.linalg.norm(NF.adjoint_nfft(x, f, 16, 2.0, 4) - ref) / np.linalg.norm(ref)
    return err < 1e-5


def _weights_pin():
    x = inputs.random_points(200, 2, 31)
    w = WT.weights(x, 4)
    A = FO.matrix_A(x, 4)
    return np.max(np.abs(np.conj(A).T @ (w[:, None] * A) - np.eye(16))) < 1e-10


def test_pins_hold_unpatched():
    assert _nfft_pin() and _weights_pin()


MUTANTS = {
    "dft_sign": (NF, "_dft_axis", lambda orig: (lambda M, Ms, sign: orig(M, Ms, -sign))),
    "drop_deconvolution": (NF, "what_grid", lambda orig: (lambda *a: np.ones_like(orig(*a)))),
    "slot_offset": (NF, "point_slots", lambda orig: (lambda x, Ms, m, p=NF.PATTERN_PAPER:
                                                         (lambda c, v: (c + 1, v))(*orig(x, Ms, m, p)))),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_nfft_mutants_fail(monkeypatch, name):
    mod, attr, make = MUTANTS[name]
    monkeypatch.setattr(mod, attr, make(getattr(mod, attr)))
    assert not _nfft_pin()


WINDOW_MUTANTS = {
    "window_uses_M_not_Ms": (W._W1, lambda orig: (lambda x, M, Ms, m: orig(x, M, M, m))),
    "kb_transform_scale": (W._WHAT1, lambda orig: (lambda k, M, Ms, m: orig(k * 2, M, Ms, m))),
    "kb_transform_m_plus_1": (W._WHAT1, lambda orig: (lambda k, M, Ms, m: orig(k, M, Ms, m + 1))),
}


@pytest.mark.parametrize("name", sorted(WINDOW_MUTANTS))
def test_window_mutants_fail(monkeypatch, name):
    table, make = WINDOW_MUTANTS[name]
    monkeypatch.setitem(table, W.KB, make(table[W.KB]))
    assert not _nfft_pin()


@pytest.mark.parametrize("mutant", ["scaled_points", "wrong_e0", "degree_M"])
def test_weight_mutants_fail(monkeypatch, mutant):
    if mutant == "scaled_points":
        orig = WT.matrix_A
        monkeypatch.setattr(WT, "matrix_A", lambda x, M: orig(1.01 * x, M))
    elif mutant == "wrong_e0":
        orig = WT.e0
        monkeypatch.setattr(WT, "e0", lambda M2, d: np.roll(orig(M2, d), 1))
    else:
        orig = WT.weights
        monkeypatch.setattr(WT, "weights", lambda x, M, rcond=1e-13: orig(x, M // 2, rcond))
    assert not _weights_pin()


# --- the real-field least squares of B_opt (reading R6) --------------------------------

def _real_solve_mutant(orig, how):
    """solve_column with one plausible mistake in its real-field branch only."""
    def solve(xm, l, M, Ms, m, kind, field="complex", rcond=1e-12):
        if field != "real":
            return orig(xm, l, M, Ms, m, kind, field, rcond)
        if how == "conj_block":      # imaginary block stacked with the wrong sign
            return orig(-xm, l, M, Ms, m, kind, field, rcond)
        b, e = orig(xm, l, M, Ms, m, kind, field, rcond)
        if how == "sign":
            b = -b
        elif how == "zero":
            b = np.zeros_like(b)
        elif how == "re_of_complex":  # the real part of the complex solution
            b = orig(xm, l, M, Ms, m, kind, "complex", rcond)[0].real.astype(np.complex128)
        return b, e
    return solve


@pytest.mark.parametrize("how", ["sign", "zero", "re_of_complex", "conj_block"])
def test_real_field_mutants_fail(monkeypatch, how):
    from oracle import bopt as BO
    from tests.test_oracle_bopt import real_field_pin_holds
    assert real_field_pin_holds()
    monkeypatch.setattr(BO, "solve_column", _real_solve_mutant(BO.solve_column, how))
    assert not real_field_pin_holds()
