"""Pins of the oracle's geometry against closed forms, library routines and the paper's
worked special points (not gpu)."""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import (
    great_circle_curve,
    inverse_stereographic_projection,
    projected_circle,
    rodrigues,
    rotation_error,
    stereographic_projection,
)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _unit(rng, n):
    x = rng.standard_normal((n, 3))
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def test_projection_round_trip():
    rng = np.random.default_rng(1)
    x = _unit(rng, 2000)
    x = x[x[:, 2] < 0.99]
    uv = stereographic_projection(x)
    back = inverse_stereographic_projection(uv[:, 0], uv[:, 1])
    assert np.max(np.abs(back - x)) < 1e-12
    uv2 = rng.uniform(-3, 3, size=(2000, 2))
    x2 = inverse_stereographic_projection(uv2[:, 0], uv2[:, 1])
    assert np.max(np.abs(np.linalg.norm(x2, axis=1) - 1.0)) < 1e-14
    assert np.max(np.abs(stereographic_projection(x2) - uv2)) < 1e-12


def test_projection_golden_points():
    """Points fixed by Eqs. 11-12 (tests/golden/projection_points.txt, derived by hand)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "projection_points.txt"))
    for a, b, c, A, B in rows:
        uv = stereographic_projection([a, b, c])
        assert np.allclose(uv, [A, B], atol=1e-15)
        assert np.allclose(inverse_stereographic_projection(A, B), [a, b, c], atol=1e-15)


def test_equator_is_unit_circle_and_south_is_disk():
    rng = np.random.default_rng(2)
    t = rng.uniform(-math.pi, math.pi, 500)
    eq = np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], axis=1)
    assert np.allclose(np.linalg.norm(stereographic_projection(eq), axis=1), 1.0, atol=1e-14)
    x = _unit(rng, 1000)
    south = x[x[:, 2] < -1e-6]
    assert np.all(np.linalg.norm(stereographic_projection(south), axis=1) < 1.0)


def test_curve_is_projected_constraint():
    """F(u,v) / (1 + u^2 + v^2) = d . r(u,v): the curve is the image of r . d = 0 (Eq. 8)."""
    rng = np.random.default_rng(3)
    d = rng.standard_normal((500, 3))
    uv = rng.uniform(-2, 2, size=(500, 2))
    r = inverse_stereographic_projection(uv[:, 0], uv[:, 1])
    lhs = great_circle_curve(d, uv[:, 0], uv[:, 1]) / (1 + uv[:, 0] ** 2 + uv[:, 1] ** 2)
    rhs = np.einsum("ij,ij->i", d, r)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_great_circle_projects_onto_eq13_circle():
    """Axes orthogonal to d (built by cross products) land on F = 0 and on the circle of
    Eq. 13 with (A, B, C, D) = (d1, d2, d3, 0); its radius is |d| / |d3|."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        d = rng.standard_normal(3)
        e = np.cross(d, rng.standard_normal(3))
        e /= np.linalg.norm(e)
        f = np.cross(d, e) / np.linalg.norm(d)
        t = rng.uniform(-math.pi, math.pi, 200)
        pts = np.cos(t)[:, None] * e + np.sin(t)[:, None] * f
        pts = pts[pts[:, 2] < 0.95]
        uv = stereographic_projection(pts)
        assert np.max(np.abs(great_circle_curve(d, uv[:, 0], uv[:, 1]))) < 1e-9
        cx, cy, rho2 = projected_circle(d[0], d[1], d[2], 0.0)
        assert np.allclose((uv[:, 0] - cx) ** 2 + (uv[:, 1] - cy) ** 2, rho2, rtol=1e-9)
        assert math.isclose(math.sqrt(rho2), np.linalg.norm(d) / abs(d[2]), rel_tol=1e-12)


def test_eq13_small_circle_general_D():
    """Eq. 13 for a general plane (D != 0): projected points of the circle satisfy it."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        D = rng.uniform(-0.8, 0.8)
        centre = -D * n
        e = np.cross(n, rng.standard_normal(3))
        e /= np.linalg.norm(e)
        f = np.cross(n, e)
        rad = math.sqrt(1 - D * D)
        t = rng.uniform(-math.pi, math.pi, 100)
        pts = centre + rad * (np.cos(t)[:, None] * e + np.sin(t)[:, None] * f)
        pts = pts[pts[:, 2] < 0.95]
        if abs(n[2] + D) < 1e-3:
            continue
        uv = stereographic_projection(pts)
        cx, cy, rho2 = projected_circle(n[0], n[1], n[2], D)
        assert np.allclose((uv[:, 0] - cx) ** 2 + (uv[:, 1] - cy) ** 2, rho2, rtol=1e-8, atol=1e-10)


def test_rodrigues_matches_scipy():
    rng = np.random.default_rng(6)
    for _ in range(100):
        r = rng.standard_normal(3)
        r /= np.linalg.norm(r)
        th = rng.uniform(-math.pi, math.pi)
        assert np.allclose(rodrigues(r, th), Rotation.from_rotvec(th * r).as_matrix(), atol=1e-13)


def test_rodrigues_golden():
    """90 degrees about +z takes x to y (right-hand rule)."""
    R = rodrigues([0, 0, 1], math.pi / 2)
    assert np.allclose(R, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)


def test_rotation_error_closed_form():
    rng = np.random.default_rng(7)
    for _ in range(50):
        Rg = Rotation.random(random_state=rng).as_matrix()
        r = rng.standard_normal(3)
        r /= np.linalg.norm(r)
        a = rng.uniform(0, math.pi)
        assert math.isclose(rotation_error(Rg, Rg @ rodrigues(r, a)), a, abs_tol=1e-7)
