"""The eps-band consensus accumulator of Eq. 9 on the GPU against the FP64 oracle (gpu).

A cell counts circle i when some axis of the cell lies within |r . z_i| < eps of the pair's
great circle. The GPU result must lie within the oracle's bounds everywhere and equal its
grid wherever no decision was within 1e-6 of its threshold."""
import numpy as np
import pytest

from oracle import vote as ov
from paper_2502_06337_gb300 import synth

pytestmark = pytest.mark.gpu


def _eps_grid(P, Q, G, eps):
    import torch

    from paper_2502_06337_gb300 import binding as B

    Pt = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda()
    Qt = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32)).cuda()
    grid = torch.full((G * G,), 5, dtype=torch.int32, device="cuda")
    B.axis_vote_eps(Pt, Qt, G, eps, grid)
    torch.cuda.synchronize()
    return grid.cpu().numpy().view(np.uint32).astype(np.int64).reshape(G, G)


def _check(g, ev):
    assert np.all(g >= ev["lo"]) and np.all(g <= ev["hi"]), "outside the oracle's bounds"
    certain = ev["lo"] == ev["hi"]
    assert np.array_equal(g[certain], ev["grid"][certain])


@pytest.mark.parametrize("G,eps,n", [(16, 0.05, 300), (64, 0.01, 700), (256, 0.003, 500), (512, 0.3, 120),
                                     (512, 1e-9, 400), (64, 0.0, 333), (1024, 0.002, 150), (2048, 0.001, 40)])
def test_eps_vote_matches_oracle(lib, G, eps, n):
    prob = synth.make_problem(n, (0.4,), 0.01, seed=G + n)
    P, Q = prob.P.copy(), prob.Q.copy()
    Q[0] = P[0]  # degenerate
    Q[1] = P[1] + np.array([0.0, 0.0, 0.5], dtype=np.float32)  # the unit circle
    Q[2] = P[2] + np.array([0.3, -0.4, 0.0], dtype=np.float32)  # a line through the origin
    Q[3] = P[3] + np.array([1e-6, -2e-6, 3e-6], dtype=np.float32)  # a tiny difference
    _check(_eps_grid(P, Q, G, eps), ov.eps_axis_vote(P, Q, G, eps))


def test_eps_vote_single_circles(lib):
    rng = np.random.default_rng(80)
    for d in [np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]), np.array([0.0, -1.0, 0.0])] + \
            list(rng.standard_normal((6, 3))):
        P = np.array([[0.3, -0.1, 0.2]], dtype=np.float32)
        Q = (P - d.astype(np.float32)).astype(np.float32)
        for G, eps in ((32, 0.02), (128, 0.1)):
            _check(_eps_grid(P, Q, G, eps), ov.eps_axis_vote(P, Q, G, eps))


def test_eps_vote_at_full_size(lib):
    """n = 10^6 pairs, 512^2, eps = 0.004 (about a cell): a slice against the full oracle,
    64 cells of the whole grid against the oracle's cell-by-cell count over all pairs, and
    monotonicity in eps."""
    cfg = synth.HEADLINE
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    G, eps = 512, 0.004
    whole = _eps_grid(prob.P, prob.Q, G, eps)
    sl = slice(500_000, 500_300)
    _check(_eps_grid(prob.P[sl], prob.Q[sl], G, eps), ov.eps_axis_vote(prob.P[sl], prob.Q[sl], G, eps))
    rng = np.random.default_rng(81)
    rows, cols = rng.integers(0, G, 64), rng.integers(0, G, 64)
    cnt, lo, hi = ov.eps_cell_votes(prob.P, prob.Q, G, eps, rows, cols)
    got = whole[rows, cols]
    assert np.all(got >= lo) and np.all(got <= hi)
    assert np.array_equal(got[lo == hi], cnt[lo == hi])
    wider = _eps_grid(prob.P, prob.Q, G, 0.01)
    assert np.all(wider >= whole)


def test_eps_vote_invalid_arguments(lib):
    from paper_2502_06337_gb300 import binding as B

    assert lib.sprot_axis_vote_eps(None, None, 10, 64, 0.1, None, None) == B.E_INVAL
