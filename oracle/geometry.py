"""Geometry of the method in float64 (test infrastructure; see the package header).

Equation numbers follow the LaTeX labels of the paper: Eq. 2 is Rodrigues' formula, Eqs. 5-8
the axis-only constraint, Eq. 11 the stereographic projection, Eq. 12 its inverse, Eq. 13 the
image of a sphere circle, Eq. 16 the rotation error.
"""
from __future__ import annotations

import numpy as np


def stereographic_projection(xyz):
    """Eq. 11: a point (a, b, c) of the unit sphere maps to (A, B) = (a, b) / (1 - c).

    The projection pole is (0, 0, 1); the south pole maps to the origin and the equator to
    the unit circle. ``xyz`` is (..., 3); returns (..., 2).
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    a, b, c = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    return np.stack([a / (1.0 - c), b / (1.0 - c)], axis=-1)


def inverse_stereographic_projection(A, B):
    """Eq. 12: (A, B) maps back to (2A, 2B, A^2 + B^2 - 1) / (1 + A^2 + B^2)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    s = A * A + B * B
    return np.stack([2.0 * A, 2.0 * B, s - 1.0], axis=-1) / (1.0 + s)[..., None]


def projected_circle(A, B, C, D):
    """Eq. 13: the sphere circle {X : A X + B Y + C Z + D = 0} projects to the plane circle
    (x + A/(C+D))^2 + (y + B/(C+D))^2 = (A^2 + B^2)/(C+D)^2 + (C-D)/(C+D).

    Returns (centre_x, centre_y, radius_squared). Undefined when C + D = 0 (the circle goes
    through the pole and projects to a line).
    """
    s = C + D
    return -A / s, -B / s, (A * A + B * B) / (s * s) + (C - D) / s


def great_circle_curve(d, u, v):
    """The projected constraint curve of one correspondence.

    By Eqs. 5-8 an inlier's rotation axis r satisfies r . d = 0 with d = p - q, so the
    admissible axes form the great circle of the plane d . X = 0 (Eq. 13 with D = 0).
    Substituting Eq. 12 for X and clearing the positive denominator 1 + u^2 + v^2 gives

        F(u, v) = 2 d1 u + 2 d2 v + d3 (u^2 + v^2 - 1),

    whose zero set is the projected circle and which equals (1 + u^2 + v^2) d . r(u, v).
    """
    d = np.asarray(d, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    return 2.0 * d[..., 0] * u + 2.0 * d[..., 1] * v + d[..., 2] * (u * u + v * v - 1.0)


def skew(r):
    r = np.asarray(r, dtype=np.float64)
    return np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])


def rodrigues(r, theta):
    """Eq. 2: R = I + sin(theta) [r]_x + (1 - cos(theta)) [r]_x^2 for a unit axis r."""
    K = skew(r)
    return np.eye(3) + np.sin(theta) * K + (1.0 - np.cos(theta)) * (K @ K)


def rotation_error(R_gt, R):
    """Eq. 16: e_rot = arccos(0.5 (Tr(R_gt^T R) - 1)) in radians (argument clamped to
    [-1, 1] against rounding)."""
    c = 0.5 * (np.trace(np.asarray(R_gt, dtype=np.float64).T @ np.asarray(R, dtype=np.float64)) - 1.0)
    return float(np.arccos(np.clip(c, -1.0, 1.0)))
