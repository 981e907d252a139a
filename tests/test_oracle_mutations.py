"""Planted mistakes in the oracle (CPU only) must be caught by its pins.

Each test patches one plausible slip into the oracle module (a dropped
factor, a wrong sign, a swapped operand) and checks that the brute-force
addition-theorem pin or the 2*pi weight identity no longer holds.
"""

import math

import numpy as np
import pytest

from oracle import yinyang
from paper_1806_04593_gb300 import inputs

from . import bruteforce as bf

TARGETS = [("yin", 31, 3, 10), ("yang", 20, 8, 40), ("yin", 12, 14, 25), ("yang", 5, 0, 2)]


def _pin_error(spec):
    g = yinyang.OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta,
                           spec.delta_phi, spec.lmax, spec.G)
    ry, rg = inputs.tiny_density(spec)
    res = g.solve(ry, rg, gradient=True)
    w = yinyang.overlap_weights(*yinyang.angular_edges(spec.n_theta, spec.n_phi, spec.delta_theta,
                                                       spec.delta_phi), spec.delta_theta, spec.delta_phi)
    phi_bf, g_bf = bf.potential_and_gradient(spec, w, {"yin": ry, "yang": rg}, TARGETS)
    phi_o = np.array([res["phi_" + p][n, j, k] for p, n, j, k in TARGETS])
    g_o = np.array([res["grad_" + p][:, n, j, k] for p, n, j, k in TARGETS])
    return max(np.abs(phi_bf - phi_o).max() / np.abs(phi_o).max(),
               np.abs(g_bf - g_o).max() / np.abs(g_o).max())


@pytest.fixture
def spec():
    return inputs.tiny_grid()


def test_unpatched_oracle_passes(spec):
    assert _pin_error(spec) < 1e-12


def test_dropped_factor_in_normalisation_is_caught(spec, monkeypatch):
    orig = yinyang.normalisation

    def wrong(lmax):
        N = orig(lmax)
        N[:, 1:] *= 0.5                      # forgets 2/delta^(m) for m > 0
        return N
    monkeypatch.setattr(yinyang, "normalisation", wrong)
    assert _pin_error(spec) > 1e-6


def test_swapped_cos_sin_integrals_are_caught(spec, monkeypatch):
    orig = yinyang.azimuthal_integrals
    monkeypatch.setattr(yinyang, "azimuthal_integrals", lambda L, pe: orig(L, pe)[::-1])
    assert _pin_error(spec) > 1e-6


def test_wrong_sign_in_transform_is_caught(spec, monkeypatch):
    orig = yinyang.other_patch_angles

    def wrong(theta, phi):
        t, p = orig(theta, phi)
        return t, -p
    monkeypatch.setattr(yinyang, "other_patch_angles", wrong)
    assert _pin_error(spec) > 1e-6


def test_off_by_one_radial_index_is_caught(spec, monkeypatch):
    orig = yinyang.radial_integrals

    def wrong(lmax, r):
        Rin, Rout = orig(lmax, r)
        return np.roll(Rin, 1, axis=1), Rout
    monkeypatch.setattr(yinyang, "radial_integrals", wrong)
    assert _pin_error(spec) > 1e-6


def test_wrong_derivative_identity_is_caught(spec, monkeypatch):
    orig = yinyang.dlegendre_dtheta
    monkeypatch.setattr(yinyang, "dlegendre_dtheta", lambda P: -orig(P))
    assert _pin_error(spec) > 1e-6


def test_plain_unit_weights_break_the_two_pi_identity(spec):
    te, pe = yinyang.angular_edges(spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi)
    dO = (np.cos(te[:-1]) - np.cos(te[1:]))[:, None] * (pe[1:] - pe[:-1])[None, :]
    assert abs(dO.sum() - 2 * math.pi) > 0.1        # without w the patch area exceeds 2 pi
