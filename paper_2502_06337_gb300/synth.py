"""Seeded synthetic rotation problems.

This module only draws inputs: point sets P, Q with a known ground truth. It holds none of
the estimator's arithmetic (no projection, no vote, no angle, no refinement), so both the
CUDA path and the FP64 oracle can be fed from it without sharing any method code.

The workloads follow the synthetic experiments of the paper (Sec. V-A-1): random 3-D
points, a random rotation applied to the inliers, Gaussian noise of standard deviation
sigma on the inliers, and a fraction rho of outliers drawn independently of P. Points are
drawn uniformly in the cube [-1, 1]^3 rather than normalised to unit length.

Every generator is driven by ``numpy.random.Generator(PCG64(seed))`` and returns float32
arrays in row-major n x 3 layout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation: a normalised 4-D Gaussian read as a unit quaternion."""
    w, x, y, z = rng.standard_normal(4)
    s = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / s, x / s, y / s, z / s
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
        ],
        dtype=np.float64,
    )


@dataclass
class Problem:
    """One rotation problem with its ground truth.

    ``truth[i]`` is the index of the rotation that generated q_i, or -1 for an outlier.
    """

    P: np.ndarray
    Q: np.ndarray
    rotations: list
    truth: np.ndarray
    sigma: float
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.P.shape[0])


def make_problem(
    n: int,
    inlier_fracs=(0.5,),
    sigma: float = 0.01,
    seed: int = 0,
    rotations=None,
    unit: bool = False,
) -> Problem:
    """Draw P uniform in [-1,1]^3; for each rotation a, a share ``inlier_fracs[a]`` of the
    correspondences gets q = R_a p + N(0, sigma^2 I); the rest get q uniform in [-1,1]^3.

    ``unit``: the recipe of the paper's synthetic experiments (Sec. V-A) instead: P and the
    outlier points are unit-length vectors (normalised Gaussian draws); inliers are still
    R_a p plus Gaussian noise of standard deviation sigma.

    Inlier positions are a random permutation, so inliers are not contiguous.
    """
    rng = _rng(seed)
    if unit:
        P = rng.standard_normal((n, 3))
        P /= np.linalg.norm(P, axis=1, keepdims=True)
    else:
        P = rng.uniform(-1.0, 1.0, size=(n, 3))
    if rotations is None:
        rotations = [random_rotation(rng) for _ in inlier_fracs]
    counts = [int(round(f * n)) for f in inlier_fracs]
    if sum(counts) > n:
        raise ValueError("inlier fractions exceed 1")
    truth = np.full(n, -1, dtype=np.int32)
    perm = rng.permutation(n)
    start = 0
    for a, c in enumerate(counts):
        truth[perm[start : start + c]] = a
        start += c
    if unit:
        Q = rng.standard_normal((n, 3))
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    else:
        Q = rng.uniform(-1.0, 1.0, size=(n, 3))
    noise = rng.standard_normal((n, 3)) * sigma
    for a, R in enumerate(rotations):
        m = truth == a
        Q[m] = P[m] @ np.asarray(R).T + noise[m]
    return Problem(
        P=np.ascontiguousarray(P, dtype=np.float32),
        Q=np.ascontiguousarray(Q, dtype=np.float32),
        rotations=[np.asarray(R, dtype=np.float64) for R in rotations],
        truth=truth,
        sigma=float(sigma),
        seed=int(seed),
    )


# ---------------------------------------------------------------------------------------
# The five workloads. Sizes, grids and bins are those the benchmarks are quoted on.
# ---------------------------------------------------------------------------------------

#: single rotation, n = 1000, half outliers, 256^2 grid, 360 bins
SMALL = dict(n=1000, inlier_fracs=(0.5,), sigma=0.01, grid=256, angle_bins=360, k=1)
#: single rotation at the paper's headline scale: n = 10^6, 90 % outliers, 512^2, 720 bins
HEADLINE = dict(n=1_000_000, inlier_fracs=(0.1,), sigma=0.01, grid=512, angle_bins=720, k=1)
#: three rotations owning 15 % each, 55 % outliers, top-3 with a 2 degree suppression radius
MULTI = dict(
    n=200_000, inlier_fracs=(0.15, 0.15, 0.15), sigma=0.01, grid=512, angle_bins=720, k=3,
    nms_deg=2.0,
)


def default_tau(sigma: float) -> float:
    """Residual threshold used by the workloads: 3 sigma sqrt(3), at least 0.05 (the inlier
    noise is isotropic Gaussian, so the residual norm is sigma times a chi-3 variable)."""
    return max(0.05, 3.0 * math.sqrt(3.0) * sigma)


def batch_specs(m: int = 4096, seed: int = 0, n_lo: int = 500, n_hi: int = 200_000):
    """Parameters of the batched workload: n log-uniform in [n_lo, n_hi], outlier rate
    uniform in [0.50, 0.95], noise sigma uniform in [0.001, 0.02]."""
    rng = _rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=m)).astype(np.int64)
    rho = rng.uniform(0.50, 0.95, size=m)
    sig = rng.uniform(0.001, 0.02, size=m)
    seeds = rng.integers(0, 2**31 - 1, size=m)
    return [
        dict(n=int(ns[i]), inlier_fracs=(1.0 - float(rho[i]),), sigma=float(sig[i]), seed=int(seeds[i]))
        for i in range(m)
    ]


def serve_specs(m: int, seed: int = 0, rate_hz: float = 2000.0, n_lo: int = 1000,
                n_hi: int = 1_000_000):
    """Served stream: Poisson arrivals at ``rate_hz``; n log-uniform in [n_lo, n_hi];
    outlier rate uniform in [0.50, 0.99]; 1-3 rotations sharing the inliers equally."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=m)
    t = np.cumsum(gaps)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=m)).astype(np.int64)
    rho = rng.uniform(0.50, 0.99, size=m)
    nrot = rng.integers(1, 4, size=m)
    seeds = rng.integers(0, 2**31 - 1, size=m)
    out = []
    for i in range(m):
        share = (1.0 - float(rho[i])) / int(nrot[i])
        out.append(dict(t_arrive=float(t[i]), n=int(ns[i]), inlier_fracs=(share,) * int(nrot[i]),
                        sigma=0.01, seed=int(seeds[i])))
    return out
