"""Pins of the semi-analytic ellipsoid potential (the §5 validation's
reference) against a library routine, closed forms and Poisson's equation."""

import math

import numpy as np
import pytest

from oracle import ellipsoid as el

AXES = (0.5, 0.75, 1.0)     # b = 1.5 a, c = 2 a (§5)


def test_carlson_integrals_against_scipy():
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "elliprf"):
        pytest.skip("scipy without Carlson integrals")
    rng = np.random.default_rng(1)
    x, y, z = rng.uniform(1e-3, 10.0, (3, 2000))
    assert np.abs(el.carlson_rf(x, y, z) / special.elliprf(x, y, z) - 1).max() <= 1e-14
    assert np.abs(el.carlson_rd(x, y, z) / special.elliprd(x, y, z) - 1).max() <= 1e-14
    # one argument zero (the complete integrals)
    assert abs(el.carlson_rf(0.0, 2.0, 3.0) / special.elliprf(0.0, 2.0, 3.0) - 1) <= 1e-14
    assert abs(el.carlson_rd(0.0, 2.0, 3.0) / special.elliprd(0.0, 2.0, 3.0) - 1) <= 1e-14


def test_carlson_closed_forms():
    v = np.array([0.01, 1.0, 7.5, 300.0])
    assert np.abs(el.carlson_rf(v, v, v) * np.sqrt(v) - 1).max() <= 1e-15
    assert np.abs(el.carlson_rd(v, v, v) * v ** 1.5 - 1).max() <= 1e-15
    # R_F(0, y, y) = pi / (2 sqrt(y));  R_F(x, y, y) = arccos(sqrt(x/y)) / sqrt(y - x) for x < y
    assert abs(el.carlson_rf(0.0, 4.0, 4.0) - math.pi / 4) <= 1e-15
    assert abs(el.carlson_rf(1.0, 3.0, 3.0) - math.acos(math.sqrt(1 / 3)) / math.sqrt(2)) <= 1e-15


def test_sphere_limit_inside_and_outside():
    R, G, rho0 = 0.7, 1.3, 2.0
    M = 4 * math.pi / 3 * R ** 3 * rho0
    rng = np.random.default_rng(2)
    v = rng.normal(size=(3, 500))
    v /= np.linalg.norm(v, axis=0)
    r = rng.uniform(0.0, 3.0, 500)
    phi = el.ellipsoid_potential(*(r * v), (R, R, R), rho0, G)
    ref = np.where(r <= R, -G * M * (3 * R ** 2 - r ** 2) / (2 * R ** 3), -G * M / np.maximum(r, 1e-300))
    assert np.abs(phi / ref - 1).max() <= 1e-13


def test_poisson_equation_inside_and_outside():
    """Central-difference Laplacian: 4 pi G rho0 inside, 0 outside."""
    G, rho0, h = 1.0, 1.0, 1e-3
    pts = np.array([[0.1, -0.2, 0.3], [0.2, 0.3, -0.5], [-0.3, 0.1, 0.1],      # inside
                    [0.9, 0.2, 0.4], [-0.2, 1.2, -0.6], [0.1, 0.1, 1.5]]).T     # outside
    inside = (pts[0] / AXES[0]) ** 2 + (pts[1] / AXES[1]) ** 2 + (pts[2] / AXES[2]) ** 2 <= 1
    assert inside.tolist() == [True] * 3 + [False] * 3
    phi0 = el.ellipsoid_potential(*pts, AXES, rho0, G)
    lap = np.zeros(pts.shape[1])
    for k in range(3):
        d = np.zeros((3, 1))
        d[k] = h
        lap += (el.ellipsoid_potential(*(pts + d), AXES, rho0, G)
                + el.ellipsoid_potential(*(pts - d), AXES, rho0, G) - 2 * phi0) / h ** 2
    target = np.where(inside, 4 * math.pi * G * rho0, 0.0)
    assert np.abs(lap - target).max() <= 1e-4 * 4 * math.pi


def test_continuity_across_the_surface_and_far_field():
    G, rho0 = 1.0, 1.0
    M = 4 * math.pi / 3 * np.prod(AXES) * rho0
    rng = np.random.default_rng(3)
    v = rng.normal(size=(3, 200))
    v /= np.linalg.norm(v, axis=0)
    rs = 1.0 / np.sqrt((v[0] / AXES[0]) ** 2 + (v[1] / AXES[1]) ** 2 + (v[2] / AXES[2]) ** 2)
    eps = 1e-7
    pin = el.ellipsoid_potential(*(v * rs * (1 - eps)), AXES)
    pout = el.ellipsoid_potential(*(v * rs * (1 + eps)), AXES)
    assert np.abs(pin - pout).max() <= 1e-6 * np.abs(pin).max()
    far = el.ellipsoid_potential(*(v * 1e3), AXES, rho0, G)
    assert np.abs(far / (-G * M / 1e3) - 1).max() <= 1e-6
