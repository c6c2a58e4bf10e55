"""Pins of the oracle's vote, peaks, angle vote and refinement (not gpu).

Each test checks the oracle against something other than itself: hand-derived fixtures,
an independent geometric formulation of the cell test, Algorithm 1's sampled rasteriser,
closed forms with noise-free inputs, invariances, or library routines."""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from oracle import vote as ov
from paper_2502_06337_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _single(d):
    """A one-correspondence problem whose difference p - q is d (q = 0)."""
    P = np.asarray([d], dtype=np.float32)
    Q = np.zeros_like(P)
    return P, Q


def test_golden_unit_circle():
    want = np.loadtxt(os.path.join(GOLDEN, "unit_circle_G8.txt"), dtype=np.int64)
    av = oracle.axis_vote(*_single([0, 0, 1]), 8)
    assert np.array_equal(av["grid"], want)
    assert np.array_equal(av["lo"], want) and np.array_equal(av["hi"], want)


def test_golden_line_through_pole():
    want = np.loadtxt(os.path.join(GOLDEN, "line_u0_G8.txt"), dtype=np.int64)
    av = oracle.axis_vote(*_single([1, 0, 0]), 8)
    assert np.array_equal(av["grid"], want)
    assert av["lo"].sum() == 0 and np.array_equal(av["hi"], want)


def _circle_geometry_cells(d, G):
    """Independent form of the cell test: the plane circle of centre -(d1, d2)/d3 and radius
    |d|/|d3| meets a closed box iff (nearest distance) <= radius <= (farthest distance)."""
    e = ov.grid_edges(G)
    cx, cy = -d[0] / d[2], -d[1] / d[2]
    rho = np.linalg.norm(d) / abs(d[2])
    out = np.zeros((G, G), dtype=bool)
    for i in range(G):
        for j in range(G):
            u0, u1, v0, v1 = e[j], e[j + 1], e[i], e[i + 1]
            nx = min(max(cx, u0), u1)
            ny = min(max(cy, v0), v1)
            near = math.hypot(nx - cx, ny - cy)
            far = max(math.hypot(x - cx, y - cy) for x in (u0, u1) for y in (v0, v1))
            out[i, j] = near <= rho <= far
    return out


@pytest.mark.parametrize("seed", range(6))
def test_cell_test_matches_circle_geometry(seed):
    rng = np.random.default_rng(seed)
    G = 32
    for _ in range(4):
        d = rng.standard_normal(3)
        if abs(d[2]) < 0.05:
            continue
        av = oracle.axis_vote(*_single(d), G)
        geo = _circle_geometry_cells(d, G)
        certain = av["lo"] == av["hi"]
        assert np.array_equal(av["grid"].astype(bool)[certain], geo[certain])
        assert certain.mean() > 0.99


@pytest.mark.parametrize("seed", range(4))
def test_algorithm1_sampled_cells_are_voted(seed):
    """Every cell hit by Algorithm 1's sampled circle is voted, and with dense sampling the
    two sets coincide up to cells the curve only grazes."""
    rng = np.random.default_rng(100 + seed)
    G = 64
    for _ in range(3):
        d = rng.standard_normal(3)
        av = oracle.axis_vote(*_single(d), G)
        voted = set(zip(*np.nonzero(av["grid"])))
        hit = ov.sampled_circle_cells(d, G, 400_000)
        assert hit <= voted
        missed = voted - hit
        assert len(missed) <= max(2, 0.01 * len(voted))


def test_line_cells_and_symmetry():
    G = 16
    av = oracle.axis_vote(*_single([0, 1, 0]), G)  # the line v = 0: rows 7 and 8
    want = np.zeros((G, G), dtype=np.int64)
    want[G // 2 - 1 : G // 2 + 1, :] = 1
    assert np.array_equal(av["grid"], want)


def test_cell_count_sum_and_degenerate():
    prob = synth.make_problem(200, (0.5,), 0.01, seed=3)
    P, Q = prob.P.copy(), prob.Q.copy()
    Q[:5] = P[:5]  # five exact degenerate pairs
    G = 32
    av = oracle.axis_vote(P, Q, G)
    assert av["n_degenerate"] == 5
    total = 0
    for i in range(5, 200):
        Fmin, Fmax = ov.circle_cell_extrema(P[i].astype(np.float64) - Q[i], G)
        total += int(((Fmin <= 0) & (Fmax >= 0)).sum())
    assert av["grid"].sum() == total


def test_noise_free_axis_cell_gets_every_vote():
    """sigma = 0: every inlier circle passes through the true axis, so the cell holding the
    projected axis gets one vote per pair and is the peak (Fig. 3a)."""
    for seed in range(4):
        prob = synth.make_problem(300, (1.0,), 0.0, seed=seed)
        R = prob.rotations[0]
        rv = Rotation.from_matrix(R).as_rotvec()
        r = rv / np.linalg.norm(rv)
        if r[2] > 0:
            r = -r
        A, B = oracle.stereographic_projection(r)
        G = 64
        col, row = int((A + 1) * G / 2), int((B + 1) * G / 2)
        av = oracle.axis_vote(prob.P, prob.Q, G)
        nondeg = prob.n - av["n_degenerate"]
        assert av["grid"][row, col] == nondeg
        assert av["grid"].max() == nondeg


def test_peak_tie_break():
    g = np.zeros((4, 4), dtype=np.int64)
    g[2, 1] = 5
    g[1, 3] = 5
    assert oracle.peak_cell(g) == (1, 3, 5)


def test_top_k_suppression_by_construction():
    G = 256  # near the centre one cell spans about 0.9 degrees
    g = np.zeros((G, G), dtype=np.int64)
    g[128, 128] = 100  # peak 1
    g[128, 129] = 90   # neighbour of peak 1: within 2 degrees, suppressed
    g[129, 128] = 80
    g[40, 200] = 70    # far away: peak 2
    g[40, 201] = 69    # neighbour of peak 2
    g[200, 20] = 60    # peak 3
    peaks = oracle.top_k_cells(g, 3, 2.0)
    assert peaks == [(128, 128, 100), (40, 200, 70), (200, 20, 60)]
    # without suppression the neighbours of a peak are still no peaks of their own
    assert oracle.top_k_cells(g, 3, 0.0) == [(128, 128, 100), (40, 200, 70), (200, 20, 60)]
    assert oracle.top_k_cells(np.zeros((8, 8), dtype=np.int64), 2, 2.0) == []


def _local_maxima_by_loops(g):
    """Peaks by their definition, one cell at a time: no neighbour (8-neighbourhood, inside
    the grid) has a larger count, or an equal count at a smaller row-major index."""
    G0, G1 = g.shape
    out = np.zeros(g.shape, dtype=bool)
    for r in range(G0):
        for c in range(G1):
            ok = True
            for rr in range(r - 1, r + 2):
                for cc in range(c - 1, c + 2):
                    if (rr, cc) == (r, c) or not (0 <= rr < G0 and 0 <= cc < G1):
                        continue
                    if g[rr, cc] > g[r, c] or (g[rr, cc] == g[r, c] and rr * G1 + cc < r * G1 + c):
                        ok = False
            out[r, c] = ok
    return out


@pytest.mark.parametrize("seed", range(6))
def test_local_maxima_brute_force(seed):
    """The shifted-array form of the peak test equals the cell-by-cell definition, on small
    grids with many ties (counts 0-3) so that plateaus and grid borders are exercised."""
    rng = np.random.default_rng(seed)
    g = rng.integers(0, 4, size=(9, 9)).astype(np.int64)
    assert np.array_equal(oracle.local_maxima(g), _local_maxima_by_loops(g))


def test_local_maxima_plateau_and_border():
    g = np.zeros((6, 6), dtype=np.int64)
    g[2, 2] = g[2, 3] = 7  # a two-cell plateau: the smaller index is the peak
    g[5, 5] = 3            # a corner cell with lower neighbours
    m = oracle.local_maxima(g)
    assert m[2, 2] and not m[2, 3] and m[5, 5]
    # zero cells away from the plateau are peaks of the key too (their count is 0, never taken)
    assert oracle.top_k_cells(g, 5, 0.0) == [(2, 2, 7), (5, 5, 3)]


def test_top_k_skips_the_shoulder_of_a_larger_peak():
    """A cell on the flank of a large peak, outside the suppression radius, outranks a
    smaller peak of its own; the flank cell is no peak (Sec. IV-D takes the axes at the
    accumulator's peaks), so the smaller peak is the second axis."""
    G = 256  # near the centre a cell spans about 0.9 degrees, so 3 cells lie beyond 2 degrees
    g = np.zeros((G, G), dtype=np.int64)
    for dc, cnt in enumerate([100, 90, 75, 60, 45, 30]):
        g[128, 128 + dc] = cnt  # peak and its descending flank
    g[40, 200] = 50             # a separate, smaller peak
    assert oracle.top_k_cells(g, 2, 2.0) == [(128, 128, 100), (40, 200, 50)]
    # the flank cell 3 columns out is beyond the radius, but it is not a peak
    assert ov.axis_angle_deg(oracle.cell_axis(G, 128, 128), oracle.cell_axis(G, 128, 131)) > 2.0
    assert not oracle.local_maxima(g)[128, 131]


def test_top_k_suppresses_antipodal_axis():
    """Axis lines: a corner cell outside the unit disk and the disk cell of the opposite
    direction are one axis, so the second is suppressed."""
    G = 64
    g = np.zeros((G, G), dtype=np.int64)
    g[0, 0] = 50  # corner, centre (-63/64, -63/64): northern hemisphere
    r = oracle.inverse_stereographic_projection(-1 + 1 / G, -1 + 1 / G)
    A, B = oracle.stereographic_projection(-r)
    col, row = int((A + 1) * G / 2), int((B + 1) * G / 2)
    g[row, col] = 40
    peaks = oracle.top_k_cells(g, 2, 2.0)
    assert peaks == [(0, 0, 50)]


def test_cell_axis_is_south_and_unit():
    for G in (16, 64):
        for row in range(0, G, 5):
            for col in range(0, G, 7):
                r = oracle.cell_axis(G, row, col)
                assert abs(np.linalg.norm(r) - 1) < 1e-14 and r[2] <= 0


def test_pair_angles_closed_form():
    """q = R(r, theta) p exactly: the per-pair angle is theta for every p off the axis,
    with the sign convention of Eq. 2."""
    rng = np.random.default_rng(9)
    for _ in range(30):
        r = rng.standard_normal(3)
        r /= np.linalg.norm(r)
        th = rng.uniform(-math.pi + 1e-3, math.pi - 1e-3)
        P = rng.uniform(-1, 1, (100, 3))
        Q = P @ oracle.rodrigues(r, th).T
        ang, nb, ng = ov.pair_angles(r, P, Q)
        assert np.allclose(ang, th, atol=1e-10)
        ang2, _, _ = ov.pair_angles(-r, P, Q)
        assert np.allclose(ang2, -th, atol=1e-10)


def test_angle_bins_by_construction():
    """Pairs built at chosen angles fall in the bins the bin rule gives by hand."""
    J = 8  # bins of 45 degrees starting at -180
    r = np.array([0.0, 0.0, -1.0])
    want_deg = [-170, -100, -1, 1, 44, 46, 170]
    want_bin = [0, 1, 3, 4, 4, 5, 7]
    P = np.tile([[1.0, 0.0, 0.3]], (len(want_deg), 1))
    Q = np.stack([oracle.rodrigues(r, math.radians(a)) @ P[0] for a in want_deg])
    gate = np.ones(len(P), dtype=bool)
    av = oracle.angle_vote(P, Q, r, gate, np.zeros_like(gate), J)
    assert av["bin"].tolist() == want_bin
    assert av["hist"].tolist() == [1, 1, 0, 1, 2, 1, 0, 1]
    b, th = oracle.angle_peak(av["hist"])
    assert b == 4 and math.isclose(th, math.radians(22.5))


def test_window_gate_matches_cells():
    """The gate is the closed-box test on the window, i.e. 'some cell of the window voted'."""
    prob = synth.make_problem(150, (0.5,), 0.01, seed=11)
    G = 32
    for (row, col, w) in [(10, 12, 1), (0, 0, 1), (31, 5, 2), (16, 16, 0)]:
        gate, flag = oracle.window_gate(prob.P, prob.Q, G, row, col, w)
        r0, r1 = max(0, row - w), min(G - 1, row + w)
        c0, c1 = max(0, col - w), min(G - 1, col + w)
        for i in range(prob.n):
            d = prob.P[i].astype(np.float64) - prob.Q[i]
            Fmin, Fmax = ov.circle_cell_extrema(d, G)
            any_cell = bool(((Fmin <= 0) & (Fmax >= 0))[r0 : r1 + 1, c0 : c1 + 1].any())
            if not flag[i]:
                assert gate[i] == any_cell


def test_kabsch_is_optimal_and_proper():
    rng = np.random.default_rng(12)
    for _ in range(10):
        P = rng.standard_normal((40, 3))
        Q = rng.standard_normal((40, 3))
        R = oracle.kabsch(P, Q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1) < 1e-12
        M = Q.T @ P
        best = np.trace(R.T @ M)
        for S in Rotation.random(2000, random_state=rng).as_matrix():
            assert np.trace(S.T @ M) <= best + 1e-9


def test_kabsch_exact_recovery():
    rng = np.random.default_rng(13)
    R = Rotation.random(random_state=rng).as_matrix()
    P = rng.uniform(-1, 1, (50, 3))
    assert np.allclose(oracle.kabsch(P, P @ R.T), R, atol=1e-13)


@pytest.mark.parametrize("unit", [False, True])
def test_noise_free_solve_is_exact(unit):
    """sigma = 0 with outliers: the refined rotation is R_gt to rounding when no outlier
    lands within tau of R_gt p (checked; such seeds are skipped). ``unit``: the paper's
    unit-vector recipe (Sec. V-A) instead of points in the cube."""
    done = 0
    for seed in range(8):
        prob = synth.make_problem(400, (0.6,), 0.0, seed=seed, unit=unit)
        R = prob.rotations[0]
        res = np.linalg.norm(prob.Q.astype(np.float64) - prob.P @ R.T, axis=1)
        if np.any((prob.truth < 0) & (res <= 0.05)):
            continue
        out = oracle.solve(prob.P, prob.Q, G=64, J=180, tau=0.05)
        rot = out["rotations"][0]
        # float32 storage of q = R p limits the exactness to ~1e-7
        assert oracle.rotation_error(R, rot["R"]) < 1e-6
        assert np.array_equal(out["labels"] >= 0, prob.truth >= 0)
        done += 1
    assert done >= 4


def test_swap_invariance():
    """Swapping P and Q keeps every circle (d -> -d), mirrors the angle histogram
    (theta -> -theta) and transposes the rotation."""
    prob = synth.make_problem(300, (0.5,), 0.01, seed=21)
    G, J = 64, 90
    a = oracle.solve(prob.P, prob.Q, G, J)
    b = oracle.solve(prob.Q, prob.P, G, J)
    assert np.array_equal(a["axis"]["grid"], b["axis"]["grid"])
    ha = a["rotations"][0]["vote"]["hist"]
    hb = b["rotations"][0]["vote"]["hist"]
    assert np.array_equal(ha, hb[::-1])
    assert np.max(np.abs(a["rotations"][0]["R"].T - b["rotations"][0]["R"])) < 1e-12


def test_permutation_invariance():
    prob = synth.make_problem(300, (0.5,), 0.01, seed=22)
    perm = np.random.default_rng(0).permutation(300)
    G = 64
    a = oracle.axis_vote(prob.P, prob.Q, G)
    b = oracle.axis_vote(prob.P[perm], prob.Q[perm], G)
    assert np.array_equal(a["grid"], b["grid"])


def test_conjugation_equivariance():
    """Rotating both point sets by S conjugates the answer: R -> S R S^T (to the noise)."""
    prob = synth.make_problem(600, (0.5,), 0.005, seed=23)
    S = Rotation.from_rotvec([0.3, -0.2, 0.5]).as_matrix()
    a = oracle.solve(prob.P, prob.Q, 64, 180)
    Ps = (prob.P.astype(np.float64) @ S.T).astype(np.float32)
    Qs = (prob.Q.astype(np.float64) @ S.T).astype(np.float32)
    b = oracle.solve(Ps, Qs, 64, 180)
    Ra = a["rotations"][0]["R"]
    Rb = b["rotations"][0]["R"]
    assert oracle.rotation_error(S @ Ra @ S.T, Rb) < 2e-3


def test_small_workload_accuracy():
    """The 1000-pair, 50 % outlier workload: the refined rotation is within noise of R_gt."""
    cfg = synth.SMALL
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    out = oracle.solve(prob.P, prob.Q, cfg["grid"], cfg["angle_bins"], tau=synth.default_tau(0.01))
    err = oracle.rotation_error(prob.rotations[0], out["rotations"][0]["R"])
    assert err < math.radians(0.2)
    # the vote rotation itself is within a couple of cells / bins
    assert oracle.rotation_error(prob.rotations[0], out["rotations"][0]["R_vote"]) < math.radians(3)


def test_two_rotations_give_two_peaks():
    """Fig. 3d-f: with two rotations the accumulator has two peaks, one per axis."""
    prob = synth.make_problem(1200, (0.35, 0.35), 0.005, seed=31)
    out = oracle.solve(prob.P, prob.Q, G=64, J=180, k=2, nms_deg=4.0, tau=0.05)
    assert len(out["rotations"]) == 2
    errs = sorted(
        min(oracle.rotation_error(Rg, x["R"]) for x in out["rotations"]) for Rg in prob.rotations
    )
    assert errs[-1] < math.radians(0.5)


def test_golden_small_regression():
    """Fixture written by tests/golden/make_golden.py (oracle only)."""
    import json

    with open(os.path.join(GOLDEN, "small_seed0.json")) as f:
        g = json.load(f)
    cfg = synth.SMALL
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    out = oracle.solve(prob.P, prob.Q, cfg["grid"], cfg["angle_bins"], tau=g["tau"])
    rot = out["rotations"][0]
    assert list(rot["cell"]) == g["cell"]
    assert rot["axis_votes"] == g["axis_votes"]
    assert rot["bin"] == g["bin"]
    assert int(out["labels"].__ge__(0).sum()) == g["n_inliers"]
    assert np.allclose(rot["R"], np.array(g["R"]), atol=1e-12)


@pytest.mark.parametrize("swap", [False, True])
def test_cap_between_corners_is_voted(swap):
    """A cell that the circle enters only with its topmost point, between the two corners of
    its bottom edge: all four corners lie outside the circle, yet the point (0.125, 0.251) of
    the curve is inside the cell, so the cell is voted. Built by hand for G = 8: centre
    (0.125, -x) and radius sqrt(0.125^2 + x^2 + 1) with x = (1.015625 - 0.251^2) / 0.502 put
    the top of the circle at v = 0.251 (row 5 spans [0.25, 0.5], column 4 spans [0, 0.25]).
    The swapped case is the same with u and v exchanged (the leftmost-point case)."""
    x = (1.015625 - 0.251 ** 2) / 0.502
    d = np.array([-0.125, x, 1.0])
    row, col = 5, 4
    if swap:
        d = d[[1, 0, 2]]
        row, col = col, row
    assert abs(oracle.great_circle_curve(d, *((0.251, 0.125) if swap else (0.125, 0.251)))) < 1e-12
    G = 8
    e = ov.grid_edges(G)
    corners = [oracle.great_circle_curve(d, e[col + a], e[row + b]) for a in (0, 1) for b in (0, 1)]
    assert min(corners) > 0  # every corner outside
    Fmin, Fmax = ov.circle_cell_extrema(d, G)
    assert Fmin[row, col] < -1e-3 and Fmax[row, col] > 0
    av = oracle.axis_vote(np.asarray([d], np.float32), np.zeros((1, 3), np.float32), G)
    assert av["grid"][row, col] == 1 and av["lo"][row, col] == 1


# ---------------------------------------------------------------------------------------
# Algorithm 1's sampled accumulator (the literal J-point rasteriser)
# ---------------------------------------------------------------------------------------

def test_sample_basis_spans_the_great_circle():
    rng = np.random.default_rng(40)
    for d in list(rng.standard_normal((20, 3))) + [np.array([0.0, 0.0, 2.5]), np.array([0.0, 0.0, -1.0])]:
        a1, a2, na = ov.sample_basis(d)
        z = d / np.linalg.norm(d)
        for v in (a1, a2):
            assert abs(np.linalg.norm(v) - 1.0) < 1e-14 and abs(v @ z) < 1e-14
        assert abs(a1 @ a2) < 1e-14 and na > 0


def test_sampled_unit_circle_closed_form():
    """z = e3 (the equator, i.e. the unit circle of the plane): alpha0 = e1, alpha1 = e1,
    alpha2 = e1 x e3 = -e2, so sample j is (cos t_j, -sin t_j) in the plane; each cell's count
    is the number of angles whose point lies in it (several per cell: double votes)."""
    P = np.array([[0.3, -0.2, 1.5]], dtype=np.float32)
    Q = np.array([[0.3, -0.2, 0.5]], dtype=np.float32)  # d = (0, 0, 1)
    for G, J in ((4, 7), (8, 90), (2, 720)):
        got = ov.sampled_axis_vote(P, Q, G, J)
        want = np.zeros((G, G), dtype=np.int64)
        for j in range(J):
            t = -math.pi + 2.0 * math.pi * j / J
            u, v = math.cos(t), -math.sin(t)
            if abs(u) < 1.0 and abs(v) < 1.0:
                want[int(math.floor((v + 1.0) * G / 2)), int(math.floor((u + 1.0) * G / 2))] += 1
        assert np.array_equal(got["grid"], want)
        assert want.max() > 1 or J < G * 4  # several samples share a cell


def test_sampled_cells_lie_on_the_predicate_cells():
    """Every sample that is not near an edge lands in a cell the closed-cell test votes."""
    prob = synth.make_problem(40, (0.5,), 0.01, seed=41)
    G = 32
    for i in range(prob.n):
        P1, Q1 = prob.P[i:i + 1], prob.Q[i:i + 1]
        sv = ov.sampled_axis_vote(P1, Q1, G, 500)
        av = oracle.axis_vote(P1, Q1, G)
        assert np.all((sv["lo"] == 0) | (av["hi"] > 0))


def test_sampled_swap_invariance():
    """Swapping P and Q negates z: alpha1 is unchanged, alpha2 flips, and the angle set
    {t_j} is symmetric under t -> -t, so the same points are drawn."""
    prob = synth.make_problem(60, (0.4,), 0.01, seed=42)
    a = ov.sampled_axis_vote(prob.P, prob.Q, 64, 180)
    b = ov.sampled_axis_vote(prob.Q, prob.P, 64, 180)
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])


# ---------------------------------------------------------------------------------------
# Least-squares axis (Eq. 10)
# ---------------------------------------------------------------------------------------

def test_ls_axis_noise_free_is_the_rotation_axis():
    """Every noise-free inlier has z . r = 0 for the true axis r (Eq. 8), so the smallest
    eigenvalue of S is 0 and its eigenvector is r (up to sign)."""
    rng = np.random.default_rng(60)
    for _ in range(5):
        prob = synth.make_problem(400, (1.0,), 0.0, seed=int(rng.integers(1 << 30)))
        R = prob.rotations[0]
        w, V = np.linalg.eig(R)
        r_true = np.real(V[:, np.argmin(np.abs(w - 1.0))])
        got = ov.ls_axis(prob.P, prob.Q, hint=r_true)
        assert got["lam"] < 1e-9
        assert np.linalg.norm(got["axis"] - r_true / np.linalg.norm(r_true)) < 1e-6


def test_ls_axis_matches_singular_vector_of_stacked_constraints():
    """The same axis from the stacked system of Eq. 10 by SVD (right singular vector of the
    smallest singular value), with outliers and noise."""
    prob = synth.make_problem(500, (0.6,), 0.02, seed=61)
    sel = prob.truth == 0
    got = ov.ls_axis(prob.P, prob.Q, sel)
    D = prob.P[sel].astype(np.float64) - prob.Q[sel].astype(np.float64)
    Z = D / np.linalg.norm(D, axis=1, keepdims=True)
    _, sv, Vt = np.linalg.svd(Z)
    r = Vt[-1]
    r = r if r @ got["axis"] >= 0 else -r
    assert np.linalg.norm(r - got["axis"]) < 1e-9
    assert abs(sv[-1] ** 2 - got["lam"]) < 1e-9 * sv[0] ** 2


def test_ls_axis_is_equivariant_and_needs_two_directions():
    prob = synth.make_problem(300, (1.0,), 0.01, seed=62)
    S = synth.random_rotation(np.random.default_rng(63))
    a = ov.ls_axis(prob.P, prob.Q)
    b = ov.ls_axis((prob.P.astype(np.float64) @ S.T), (prob.Q.astype(np.float64) @ S.T), hint=S @ a["axis"])
    assert np.linalg.norm(b["axis"] - S @ a["axis"]) < 1e-9
    one = ov.ls_axis(prob.P[:1], prob.Q[:1])
    assert one["axis"] is None


# ---------------------------------------------------------------------------------------
# The eps-band consensus accumulator (Eq. 9)
# ---------------------------------------------------------------------------------------

def _annulus_cells(G, eps):
    """z = e3: |r . z| = |r_z| = |s - 1| / (s + 1) with s = u^2 + v^2 (Eq. 12), so the band is
    the open annulus (1 - eps)/(1 + eps) < s < (1 + eps)/(1 - eps); a closed cell meets it iff
    its nearest point to the origin is inside the outer circle and its farthest outside the
    inner one."""
    e = -1.0 + 2.0 * np.arange(G + 1) / G
    s_in, s_out = (1 - eps) / (1 + eps), (1 + eps) / (1 - eps)
    want = np.zeros((G, G), dtype=np.int64)
    for r in range(G):
        for c in range(G):
            u0, u1, v0, v1 = e[c], e[c + 1], e[r], e[r + 1]
            nu = 0.0 if u0 <= 0 <= u1 else min(abs(u0), abs(u1))
            nv = 0.0 if v0 <= 0 <= v1 else min(abs(v0), abs(v1))
            fu, fv = max(abs(u0), abs(u1)), max(abs(v0), abs(v1))
            want[r, c] = (nu * nu + nv * nv < s_out) and (fu * fu + fv * fv > s_in)
    return want


def test_eps_band_unit_circle_is_an_annulus():
    P = np.array([[0.2, 0.1, 0.9]], dtype=np.float32)
    Q = np.array([[0.2, 0.1, 0.4]], dtype=np.float32)  # d = (0, 0, 0.5)
    for G, eps in ((16, 0.05), (32, 0.2), (64, 0.01)):
        got = ov.eps_axis_vote(P, Q, G, eps)
        want = _annulus_cells(G, eps)
        certain = got["lo"] == got["hi"]
        assert np.array_equal(got["grid"][certain], want[certain]) and certain.mean() > 0.99


def test_eps_band_contains_sampled_band_points():
    """Dense points of each cell with |r . z| < eps (r by Eq. 12) lie only in voted cells,
    and the band grows with eps."""
    prob = synth.make_problem(6, (0.5,), 0.01, seed=70)
    G = 16
    m = 12
    t = (np.arange(m) + 0.5) / m
    for eps in (0.02, 0.1):
        for i in range(prob.n):
            P1, Q1 = prob.P[i:i + 1], prob.Q[i:i + 1]
            got = ov.eps_axis_vote(P1, Q1, G, eps)
            d = P1[0].astype(np.float64) - Q1[0]
            z = d / np.linalg.norm(d)
            for r in range(G):
                for c in range(G):
                    u = -1 + (2 * c + 2 * t[:, None] + 0 * t[None, :]) / G
                    v = -1 + (2 * r + 2 * t[None, :] + 0 * t[:, None]) / G
                    s = u * u + v * v
                    H = (2 * u * z[0] + 2 * v * z[1] + (s - 1) * z[2]) / (1 + s)
                    if np.any(np.abs(H) < eps):
                        assert got["hi"][r, c] == 1
    a = ov.eps_axis_vote(prob.P, prob.Q, 32, 0.01)
    b = ov.eps_axis_vote(prob.P, prob.Q, 32, 0.05)
    assert np.all(a["lo"] <= b["hi"])


def test_eps_band_tiny_eps_is_the_curve_test():
    """eps far below the cell size: the band cells are the closed-cell curve cells (Eq. 9
    reduces to the curve of Eq. 13 at cell resolution)."""
    prob = synth.make_problem(80, (0.5,), 0.01, seed=71)
    G = 64
    band = ov.eps_axis_vote(prob.P, prob.Q, G, 1e-9)
    curve = oracle.axis_vote(prob.P, prob.Q, G)
    both = (band["lo"] == band["hi"]) & (curve["lo"] == curve["hi"])
    assert np.array_equal(band["grid"][both], curve["grid"][both]) and both.mean() > 0.99


# ---- sub-cell peak (three-point parabola per grid axis) --------------------------------------

def test_subcell_offset_recovers_a_separable_parabola():
    """f(u, v) = 1010 - 16 (u - 1/4)^2 - 64 (v + 3/8)^2 sampled at the peak cell and its edge
    neighbours gives the integers c0 = 1000, (976, 992) along u and (984, 888) along v; a
    parabola through three samples of a parabola is that parabola, so the vertex is
    (1/4, -3/8) exactly."""
    g = np.zeros((5, 5), dtype=np.int64)
    g[2, 2] = 1000
    g[2, 1], g[2, 3] = 976, 992
    g[1, 2], g[3, 2] = 984, 888
    assert ov.subcell_offset(g, 2, 2) == (0.25, -0.375)


def test_subcell_offset_matches_polyfit_vertex():
    rng = np.random.default_rng(7)
    for _ in range(200):
        c0 = int(rng.integers(10, 1000))
        cm, cp = (int(x) for x in rng.integers(0, c0, 2))
        g = np.zeros((3, 3), dtype=np.int64)
        g[1, 1], g[1, 0], g[1, 2] = c0, cm, cp
        g[0, 1], g[2, 1] = cp, cm  # the v axis sees the same triple mirrored
        a, b, _ = np.polyfit([-1.0, 0.0, 1.0], [cm, c0, cp], 2)
        want = float(np.clip(-b / (2.0 * a), -0.5, 0.5))
        du, dv = ov.subcell_offset(g, 1, 1)
        assert abs(du - want) < 1e-12 and abs(dv + want) < 1e-12


def test_subcell_offset_special_cases():
    g = np.zeros((4, 4), dtype=np.int64)
    g[1, 1] = 10
    g[1, 0] = g[1, 2] = 6  # symmetric along u
    g[0, 1] = 10           # flat towards v = -1: vertex on the cell edge
    assert ov.subcell_offset(g, 1, 1) == (0.0, -0.5)
    g[0, 1] = 12           # a larger neighbour (an NMS peak next to a suppressed cell): clamped
    assert ov.subcell_offset(g, 1, 1)[1] == -0.5
    f = np.full((4, 4), 3, dtype=np.int64)
    assert ov.subcell_offset(f, 1, 2) == (0.0, 0.0)  # flat: no downward parabola
    b = np.zeros((4, 4), dtype=np.int64)
    b[0, 3], b[0, 2], b[1, 3] = 9, 5, 1
    assert ov.subcell_offset(b, 0, 3) == (0.0, 0.0)  # corner cell: a neighbour is missing on both axes


def test_subcell_axis_edges_and_centre():
    """Zero offset is the cell-centre axis; half a cell towards a neighbour is the midpoint
    of the shared edge, reached from either cell."""
    G = 32
    for row, col in [(3, 7), (16, 16), (30, 1)]:
        assert np.allclose(ov.subcell_axis(G, row, col, 0.0, 0.0), ov.cell_axis(G, row, col), atol=1e-15)
        assert np.allclose(ov.subcell_axis(G, row, col, 0.5, 0.0), ov.subcell_axis(G, row, col + 1, -0.5, 0.0),
                           atol=1e-15)
        assert np.allclose(ov.subcell_axis(G, row, col, 0.0, -0.5), ov.subcell_axis(G, row - 1, col, 0.0, 0.5),
                           atol=1e-15)
        r = ov.subcell_axis(G, row, col, 0.3, -0.2)
        assert abs(np.linalg.norm(r) - 1.0) < 1e-15 and r[2] <= 0.0


def test_subcell_axis_is_closer_to_the_true_axis():
    """Noise-free problems with outliers: over many random rotations the sub-cell axis lies
    closer to the true axis than the peak cell's centre (a wrong sign or axis would move it
    away)."""
    G = 64
    centre, sub, better = [], [], 0
    for seed in range(16):
        prob = synth.make_problem(3000, (0.5,), 0.0, seed=100 + seed)
        out = ov.solve(prob.P, prob.Q, G, 360, subcell=True)
        row, col = out["peaks"][0][:2]
        rv = Rotation.from_matrix(prob.rotations[0]).as_rotvec()
        r_true = rv / np.linalg.norm(rv)
        e0 = ov.axis_angle_deg(ov.cell_axis(G, row, col), r_true)
        e1 = ov.axis_angle_deg(out["rotations"][0]["r_cell"], r_true)
        centre.append(e0)
        sub.append(e1)
        better += e1 < e0
    assert np.mean(sub) < 0.6 * np.mean(centre)
    assert better >= 12


# ---- per-cell evaluators, vote set, labels, skew ----------------------------------------

def _mixed_pairs(n, seed):
    prob = synth.make_problem(n, (0.4,), 0.01, seed=seed)
    P, Q = prob.P.copy(), prob.Q.copy()
    Q[0] = P[0]                                              # degenerate
    Q[1] = P[1] + np.array([0.0, 0.0, 0.5], np.float32)      # the unit circle
    Q[2] = P[2] + np.array([0.3, -0.4, 0.0], np.float32)     # a line through the origin
    return P, Q


def test_cell_votes_equal_the_whole_grid():
    """cell_votes loops over cells (all circles at once); axis_vote loops over circles (all
    cells at once): on every cell of a 32 x 32 grid they must agree, bounds included."""
    P, Q = _mixed_pairs(300, 90)
    G = 32
    av = ov.axis_vote(P, Q, G)
    rows, cols = np.divmod(np.arange(G * G), G)
    cnt, lo, hi = ov.cell_votes(P, Q, G, rows, cols)
    assert np.array_equal(cnt, av["grid"].ravel())
    assert np.array_equal(lo, av["lo"].ravel()) and np.array_equal(hi, av["hi"].ravel())


def test_row_votes_equal_the_whole_grid():
    """The row-at-a-time evaluator (used on whole rows of the 10^6-pair accumulator) equals
    the whole-grid accumulator on every row, bounds included, also with chunks smaller than
    the pair count and degenerate pairs present."""
    prob = synth.make_problem(300, (0.5,), 0.01, seed=12)
    P, Q = prob.P.copy(), prob.Q.copy()
    Q[7] = P[7]  # a degenerate pair
    G = 32
    av = oracle.axis_vote(P, Q, G)
    for row in range(G):
        cnt, lo, hi = oracle.row_votes(P, Q, G, row, chunk=77)
        assert np.array_equal(cnt, av["grid"][row])
        assert np.array_equal(lo, av["lo"][row]) and np.array_equal(hi, av["hi"][row])


def test_eps_cell_votes_equal_the_whole_grid():
    P, Q = _mixed_pairs(120, 91)
    G, eps = 32, 0.03
    ev = ov.eps_axis_vote(P, Q, G, eps)
    rows, cols = np.divmod(np.arange(G * G), G)
    cnt, lo, hi = ov.eps_cell_votes(P, Q, G, eps, rows, cols)
    assert np.array_equal(cnt, ev["grid"].ravel())
    assert np.array_equal(lo, ev["lo"].ravel()) and np.array_equal(hi, ev["hi"].ravel())


def test_vote_set_wraps_around_and_bounds_flagged_pairs():
    """Peak bin 0 of J = 10 with a window of 1: bins 9, 0 and 1 are in the set (circular).
    A flagged voter two bins out may belong (upper bound only); a flagged voter one bin out
    may fall out (lower bound excludes it); a non-member never belongs."""
    J = 10
    binv = np.array([0, 1, 9, 2, 8, 5, -1, 2, 1, 0])
    member = np.array([1, 1, 1, 1, 1, 1, 0, 1, 1, 0], bool)
    flag = np.array([0, 0, 0, 0, 0, 0, 0, 1, 1, 0], bool)
    av = dict(bin=binv, member=member, member_lo=member & ~flag, member_hi=member | flag, bin_flag=flag)
    V, V_lo, V_hi = ov.vote_set(av, 0, J, 1)
    assert V.tolist() == [1, 1, 1, 0, 0, 0, 0, 0, 1, 0]
    assert V_lo.tolist() == [1, 1, 1, 0, 0, 0, 0, 0, 0, 0]   # the flagged one-bin voter may fall out
    assert V_hi.tolist() == [1, 1, 1, 0, 0, 0, 0, 1, 1, 0]   # the flagged two-bin voter may come in
    assert np.all(V_lo <= V) and np.all(V <= V_hi)


def test_assign_labels_on_constructed_pairs():
    """R_0 = I, R_1 = 90 degrees about z. Pairs fitting R_0, fitting R_1, fitting neither, and
    points on the z axis (fixed by both: residual 0 under each, so the tie goes to 0 and is
    flagged), and a pair whose residual is tau itself (flagged)."""
    rng = np.random.default_rng(92)
    R1 = Rotation.from_rotvec([0.0, 0.0, math.pi / 2]).as_matrix()
    P = rng.uniform(-1.0, 1.0, (40, 3))
    P[30:35, :2] = 0.0  # on the z axis
    Q = P.copy()
    Q[10:20] = P[10:20] @ R1.T
    Q[20:30] = P[20:30] + rng.choice([-1.0, 1.0], (10, 3)) * 0.5  # far from both
    tau = 0.05
    Q[35] = P[35] + np.array([tau, 0.0, 0.0])  # residual exactly tau under R_0
    labels, flag = ov.assign_labels(P, Q, [np.eye(3), R1], tau)
    assert np.all(labels[:10] == 0) and np.all(labels[10:20] == 1) and np.all(labels[20:30] == -1)
    assert np.all(labels[30:35] == 0) and np.all(flag[30:35])
    assert flag[35] and labels[35] in (0, -1)
    assert not flag[:30].any()


def test_skew_is_the_cross_product():
    rng = np.random.default_rng(93)
    for _ in range(20):
        r, v = rng.standard_normal(3), rng.standard_normal(3)
        assert np.allclose(oracle.geometry.skew(r) @ v, np.cross(r, v), atol=1e-15)
