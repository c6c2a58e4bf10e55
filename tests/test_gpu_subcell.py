"""The sub-cell peak axis (SPROT_SUBCELL_AXIS) on the GPU against the FP64 oracle (gpu).

Along each grid axis the peak moves to the vertex of the parabola through the counts of the
peak cell and its edge neighbours. The offsets are computed from integer counts with one
correctly rounded quotient on both sides, so on the same grid they are equal bit for bit;
the angle vote, R_vote and the refinement then follow the sub-cell axis, checked stage by
stage like the cell-centre path."""
import math

import numpy as np
import pytest

import oracle
from oracle import geometry as og
from paper_2502_06337_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(3))
def test_subcell_small_workload_parity(lib, seed):
    cfg = synth.SMALL
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=seed)
    G, J, tau = cfg["grid"], cfg["angle_bins"], synth.default_tau(cfg["sigma"])
    g = parity.run_gpu(prob.P, prob.Q, G, J, tau=tau, subcell=True)
    av = oracle.axis_vote(prob.P, prob.Q, G)
    parity.check_solve(prob.P, prob.Q, g, G, J, tau=tau, av=av, subcell=True)
    ref = oracle.solve(prob.P, prob.Q, G, J, tau=tau, grid=av["grid"], subcell=True)
    assert g["rots"][0]["cell_offset"] == ref["rotations"][0]["cell_offset"]
    assert oracle.rotation_error(ref["rotations"][0]["R"], g["rots"][0]["R"]) < parity.E2E_ROT_TOL


def test_offsets_reported_without_the_flag(lib):
    """Without the flag the axis is the cell centre, and the offsets are still reported."""
    prob = synth.make_problem(5000, (0.3,), 0.01, seed=41)
    g = parity.run_gpu(prob.P, prob.Q, 128, 360)
    parity.check_solve(prob.P, prob.Q, g, 128, 360)  # asserts the cell-centre axis and the offsets
    assert any(x != 0.0 for x in g["rots"][0]["cell_offset"])


def test_subcell_multi_rotation_parity(lib):
    prob = synth.make_problem(20000, (0.2, 0.2, 0.2), 0.01, seed=42)
    g = parity.run_gpu(prob.P, prob.Q, 256, 360, k=3, nms=2.0, subcell=True)
    assert len(g["rots"]) == 3
    parity.check_solve(prob.P, prob.Q, g, 256, 360, k=3, nms=2.0, subcell=True)


def test_subcell_many_peaks_on_a_small_grid(lib):
    """k = 8 (the maximum) on a 16 x 16 grid with two rotations and a 10-degree radius:
    suppressed neighbours can exceed a later peak, so clamped offsets occur."""
    prob = synth.make_problem(3000, (0.3, 0.3), 0.01, seed=45)
    g = parity.run_gpu(prob.P, prob.Q, 16, 90, k=8, nms=10.0, subcell=True)
    assert 2 <= len(g["rots"]) <= 8
    parity.check_solve(prob.P, prob.Q, g, 16, 90, k=8, nms=10.0, subcell=True)


def test_subcell_peak_on_the_grid_border(lib):
    """A noise-free problem whose axis projects into row 0 (v within the first cell): the peak
    lies on the lower border, so the v offset is 0 and the u offset is the oracle's. Every
    border point has |(u, v)| >= 1, so the opposite axis -r projects inside the square onto
    the same circles and ties; its row is above 0, so the tie goes to the border cell."""
    G, n = 64, 400
    u, v = 0.31, -1.0 + 0.6 * 2.0 / G
    r = np.asarray(og.inverse_stereographic_projection(u, v))
    R = og.rodrigues(r / np.linalg.norm(r), 0.7)
    rng = np.random.default_rng(43)
    P = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    Q = (P.astype(np.float64) @ R.T).astype(np.float32)
    g = parity.run_gpu(P, Q, G, 360, tau=0.01, subcell=True)
    rot = g["rots"][0]
    assert rot["cell"][0] == 0 and rot["axis_votes"] == n
    assert rot["cell_offset"][1] == 0.0
    parity.check_solve(P, Q, g, G, 360, tau=0.01, subcell=True)


def test_subcell_headline_scale(lib):
    """n = 10^6, 512^2, 720 bins with the sub-cell axis: offsets equal the oracle's on the GPU
    grid, the angle stage in full against the oracle, and the final rotation as accurate as
    the cell-centre path."""
    cfg = synth.HEADLINE
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    G, J, tau = cfg["grid"], cfg["angle_bins"], synth.default_tau(cfg["sigma"])
    g = parity.run_gpu(prob.P, prob.Q, G, J, tau=tau, subcell=True)
    parity.check_solve(prob.P, prob.Q, g, G, J, tau=tau, subcell=True)
    assert oracle.rotation_error(prob.rotations[0], g["rots"][0]["R"]) < math.radians(0.05)


def test_unknown_flags_are_rejected(lib):
    from paper_2502_06337_gb300 import binding as B

    prob = synth.make_problem(100, (0.5,), 0.01, seed=44)
    import torch

    P = torch.from_numpy(prob.P).cuda()
    Q = torch.from_numpy(prob.Q).cuda()
    with pytest.raises(B.SprotError) as e:
        B.estimate_rotations(P, Q, B.make_params(grid=64, flags=0x80))
    assert e.value.status == B.E_INVAL
