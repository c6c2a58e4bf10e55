"""Algorithm 1's sampled accumulator (J points per circle, every point votes) on the GPU
against the FP64 oracle (gpu).

The oracle decides each point's cell in float64 and flags the points that lie within its
band of a cell edge; the GPU grid must lie within the oracle's bounds everywhere and equal
its grid wherever no point was flagged."""
import numpy as np
import pytest

from oracle import vote as ov
from paper_2502_06337_gb300 import synth

pytestmark = pytest.mark.gpu


def _sampled(P, Q, G, J):
    import torch

    from paper_2502_06337_gb300 import binding as B

    Pt = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda()
    Qt = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32)).cuda()
    grid = torch.full((G * G,), 7, dtype=torch.int32, device="cuda")  # overwritten, not accumulated
    B.axis_vote_sampled(Pt, Qt, G, J, grid)
    torch.cuda.synchronize()
    return grid.cpu().numpy().view(np.uint32).astype(np.int64).reshape(G, G)


def _special(prob):
    """Pairs that exercise the edge cases: degenerate, the alpha0 fallback (d = (0, 0, c)),
    a line through the origin (d3 = 0), a tiny difference, a pure z-axis difference."""
    P, Q = prob.P.copy(), prob.Q.copy()
    Q[0] = P[0]
    Q[1] = P[1] + np.array([0.0, 0.0, 0.5], dtype=np.float32)
    Q[2] = P[2] + np.array([0.3, -0.4, 0.0], dtype=np.float32)
    Q[3] = P[3] + np.array([1e-6, 2e-6, -1e-6], dtype=np.float32)
    Q[4] = P[4] - np.array([0.0, 0.0, 0.25], dtype=np.float32)
    return P, Q


def _check(g, sv):
    assert np.all(g >= sv["lo"]) and np.all(g <= sv["hi"]), "outside the oracle's bounds"
    certain = sv["lo"] == sv["hi"]
    assert np.array_equal(g[certain], sv["grid"][certain])


@pytest.mark.parametrize("G,J,n", [(16, 90, 300), (64, 360, 1000), (256, 720, 1500), (512, 360, 777),
                                   (2048, 64, 200)])
def test_sampled_vote_matches_oracle(lib, G, J, n):
    prob = synth.make_problem(n, (0.3,), 0.01, seed=G + J)
    P, Q = _special(prob)
    g = _sampled(P, Q, G, J)
    sv = ov.sampled_axis_vote(P, Q, G, J)
    _check(g, sv)


def test_sampled_vote_single_circles(lib):
    """One pair at a time: the unit circle (d = e3), lines, and random circles."""
    rng = np.random.default_rng(50)
    G, J = 32, 1000
    for d in [np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]), np.array([0.6, -0.8, 0.0])] + \
            list(rng.standard_normal((5, 3))):
        P = np.array([[0.1, 0.2, 0.3]], dtype=np.float32)
        Q = (P - d.astype(np.float32)).astype(np.float32)
        _check(_sampled(P, Q, G, J), ov.sampled_axis_vote(P, Q, G, J))


def test_sampled_vote_at_full_size(lib):
    """n = 10^6 pairs, 512^2 grid, 360 points per circle: permuting the pairs leaves the grid
    bit-identical, the grid of two halves sums to the whole, and a 2000-pair slice of the same
    problem matches the oracle."""
    cfg = synth.HEADLINE
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    G, J = 512, 360
    whole = _sampled(prob.P, prob.Q, G, J)
    perm = np.random.default_rng(51).permutation(prob.n)
    assert np.array_equal(_sampled(prob.P[perm], prob.Q[perm], G, J), whole)
    h = prob.n // 2
    assert np.array_equal(_sampled(prob.P[:h], prob.Q[:h], G, J) + _sampled(prob.P[h:], prob.Q[h:], G, J), whole)
    sl = slice(123_456, 125_456)
    _check(_sampled(prob.P[sl], prob.Q[sl], G, J), ov.sampled_axis_vote(prob.P[sl], prob.Q[sl], G, J))
    assert whole.sum() > 0.2 * prob.n * J


def test_sampled_vote_invalid_arguments(lib):
    from paper_2502_06337_gb300 import binding as B

    assert lib.sprot_axis_vote_sampled(None, None, 10, 64, 90, None, None) == B.E_INVAL
