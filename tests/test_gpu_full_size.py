"""The axis vote at full size where its work split decides cells (gpu).

- Whole rows of the n = 10^6, 512^2 accumulator against the oracle's row-at-a-time count: the
  rows on both sides of every band seam of the vote's plan (where a circle's walk is clipped
  to a band), the first and last rows, and the peak row.
- The 16-bit slice counters at their limit: noise-free pairs with every circle through one
  cell, and slices of exactly 65535 circles (about 5 million pairs), so that the axis cell's counter in every slice
  reaches 65535 (Algorithm 1's accumulator; the closed form needs no oracle run: the cell of
  the true axis gets one vote from every non-degenerate pair)."""
import numpy as np
import pytest

import oracle
from paper_2502_06337_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


def test_band_seam_rows_at_full_size(lib):
    """Whole rows and columns at every band seam (the vote clips the curve's row caps to bands of
    rows and its column caps to bands of columns with the same edges), the first and last rows,
    and the peak row. A column of the accumulator of (P, Q) is the row of the accumulator of the
    pairs with their first two coordinates exchanged (F is symmetric in (u, d1) and (v, d2))."""
    from paper_2502_06337_gb300 import binding as B

    cfg = synth.HEADLINE
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    G, J = cfg["grid"], cfg["angle_bins"]
    g = parity.run_gpu(prob.P, prob.Q, G, J, tau=synth.default_tau(cfg["sigma"]))
    plan = B.vote_plan(prob.n, G)
    seams = plan["band_row0"][1:-1]
    assert len(seams) >= 1
    rows = sorted({0, G - 1, g["rots"][0]["cell"][0]} | {r for s in seams for r in (s - 1, s)})
    cols = sorted({c for s in seams for c in (s - 1, s)})
    swap = [1, 0, 2]
    lines = [(g["grid"][r], prob.P, prob.Q, r) for r in rows] + \
            [(g["grid"][:, c], prob.P[:, swap], prob.Q[:, swap], c) for c in cols]
    width = []
    for got, P, Q, k in lines:
        cnt, lo, hi = oracle.row_votes(P, Q, G, k)
        assert np.all(got >= lo) and np.all(got <= hi), k
        assert np.all(got[lo == hi] == cnt[lo == hi]), k
        width.append(hi - lo)
    # with 10^6 circles most cells have some circle within the band, but only a few: the
    # bounds stay tight (a few votes wide against thousands per cell)
    width = np.concatenate(width)
    assert width.mean() < 3 and width.max() < 40


def _noise_free(n, seed):
    prob = synth.make_problem(n, (1.0,), 0.0, seed=seed)
    r = _axis_cell(prob.rotations[0], 512)
    return prob, r


def _axis_cell(R, G):
    w, V = np.linalg.eig(np.asarray(R))
    ax = np.real(V[:, np.argmin(np.abs(w - 1.0))])
    if ax[2] > 0:
        ax = -ax
    u, v = oracle.stereographic_projection(ax)
    return int((v + 1) * G / 2), int((u + 1) * G / 2)


def test_slice_counters_at_their_limit(lib):
    import torch

    from paper_2502_06337_gb300 import binding as B

    G = 512
    # a slice count that the plan takes for exactly 65535 circles a slice (the plan rounds the
    # slices up to whole rounds of the SMs when the counters force more than one round)
    slices = next((s for s in range(48, 160) if B.vote_plan(65535 * s, G)["slices"] == s), None)
    if slices is None:
        pytest.skip("no slice count between 48 and 159 is kept exactly by this device's plan")
    n = 65535 * slices
    prob, (row, col) = _noise_free(n, seed=31)
    n_deg = int(np.sum(np.all(prob.P == prob.Q, axis=1)))
    P = torch.from_numpy(prob.P).cuda()
    Q = torch.from_numpy(prob.Q).cuda()
    grid = torch.zeros(G * G, dtype=torch.int32, device="cuda")
    B.axis_vote(P, Q, G, grid)
    torch.cuda.synchronize()
    g = grid.cpu().numpy().view(np.uint32).astype(np.int64).reshape(G, G)
    assert g[row, col] == n - n_deg
    assert g.max() == n - n_deg and int(np.argmax(g)) == row * G + col
    # sampled cells against the oracle's per-cell count (the other cells are untouched by the
    # limit but share the slices)
    rng = np.random.default_rng(5)
    rr = [row - 1, row + 1, row] + list(rng.integers(0, G, 6))
    cc = [col, col, col - 1] + list(rng.integers(0, G, 6))
    cnt, lo, hi = oracle.cell_votes(prob.P, prob.Q, G, rr, cc)
    got = g[rr, cc]
    assert np.all(got >= lo) and np.all(got <= hi)
    assert np.all(got[lo == hi] == cnt[lo == hi])
    # the whole solve, alone and as a batch instance beside a small problem (slices of at most
    # 32768 circles there): the peak is the axis cell with every vote
    prm = B.make_params(grid=G, angle_bins=360, tau=0.05)
    rot = B.estimate_rotation(P, Q, prm)
    assert tuple(rot["cell"]) == (row, col) and rot["axis_votes"] == n - n_deg
    small = synth.make_problem(5000, (0.5,), 0.01, seed=32)
    Ps, Qs = torch.from_numpy(small.P).cuda(), torch.from_numpy(small.Q).cuda()
    res, _ = B.estimate_batch([(P, Q, prm), (Ps, Qs, B.make_params(grid=256, angle_bins=360, tau=0.05))])
    assert tuple(res[0][0]["cell"]) == (row, col) and res[0][0]["axis_votes"] == n - n_deg
    assert parity.rot_diff(res[0][0]["R"], rot["R"]) < 1e-9
