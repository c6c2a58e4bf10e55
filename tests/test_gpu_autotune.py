"""The plan autotuner (gpu): its knobs change how the work is cut, never a result.

The accumulator is an exact count whatever the slicing and the item sizes, so every candidate
plan must give the default plan's grid bit for bit, the same peak cell, angle bin, inlier count
and labels, and rotations equal up to FP64 summation order (1e-9); a tuned plan on a small case
must also lie within the oracle's bounds (Algorithm 1's accumulator, Sec. IV-A)."""
import numpy as np
import pytest

import oracle
from paper_2502_06337_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu

SINGLE = [dict(vote_rounds=r, chunk_div=d, batch_slice=32768, batch_div=1200) for r in (1, 2, 3)
          for d in (300, 600, 1200)]
BATCH = [dict(vote_rounds=1, chunk_div=600, batch_slice=s, batch_div=d) for s in (16384, 32768, 65535)
         for d in (600, 1200, 2400)]


@pytest.fixture(autouse=True)
def _fresh_table(lib):
    from paper_2502_06337_gb300 import binding as B

    B.autotune_reset()
    yield
    B.autotune_reset()


def _solve(P, Q, prm):
    import torch

    from paper_2502_06337_gb300 import binding as B

    G = prm.grid
    grid = torch.zeros(G * G, dtype=torch.int32, device="cuda")
    labels = torch.zeros(P.shape[0], dtype=torch.int32, device="cuda")
    rots = B.estimate_rotations(P, Q, prm, labels=labels, debug={"grid": grid}, allow_noaxis=True)
    torch.cuda.synchronize()
    return rots, grid.cpu().numpy(), labels.cpu().numpy()


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert (x["cell"], x["bin"], x["n_inliers"], x["axis_votes"]) == (y["cell"], y["bin"], y["n_inliers"],
                                                                         y["axis_votes"])
        assert parity.rot_diff(x["R"], y["R"]) < parity.ROT_TOL


def _knob_view(k):
    return {f: k[f] for f in ("vote_rounds", "chunk_div", "batch_slice", "batch_div")}


def test_every_single_plan_gives_the_default_results(lib):
    import torch

    from paper_2502_06337_gb300 import binding as B

    prob = synth.make_problem(300_000, (0.05, 0.05), 0.01, seed=41)
    P, Q = torch.from_numpy(prob.P).cuda(), torch.from_numpy(prob.Q).cuda()
    prm = B.make_params(grid=512, angle_bins=720, k=2, tau=0.05)
    ref, g0, l0 = _solve(P, Q, prm)
    for kn in SINGLE:
        B.set_tuned_plan(prob.n, kn, G=512)
        found, used = B.tuned_plan(prob.n, 512)
        assert found and _knob_view(used) == kn
        rots, g, lab = _solve(P, Q, prm)
        assert np.array_equal(g, g0), kn
        assert np.array_equal(lab, l0), kn
        _same(rots, ref)
    # the tuner: a candidate wins, is stored for the class, and solves give the same results
    B.autotune_reset()
    win = B.autotune_plan(P, Q, prm, reps=3)
    assert _knob_view(win) in SINGLE
    assert 0 < win["ms_tuned"] <= win["ms_default"]
    found, used = B.tuned_plan(prob.n, 512)
    assert found and _knob_view(used) == _knob_view(win)
    rots, g, _ = _solve(P, Q, prm)
    assert np.array_equal(g, g0)
    _same(rots, ref)


def test_tuned_plan_within_oracle_bounds(lib):
    """A non-default plan (three rounds of slices, fine per-pair items) on a small case: the
    whole accumulator against the oracle."""
    from paper_2502_06337_gb300 import binding as B

    prob = synth.make_problem(6000, (0.3,), 0.01, seed=42)
    G = 128
    B.set_tuned_plan(prob.n, dict(vote_rounds=3, chunk_div=2400, batch_slice=32768, batch_div=1200), G=G)
    g = parity.run_gpu(prob.P, prob.Q, G, 360, tau=0.05)
    ev = oracle.axis_vote(prob.P, prob.Q, G)
    got = g["grid"].astype(np.int64)
    assert np.all(got >= ev["lo"]) and np.all(got <= ev["hi"])
    certain = ev["lo"] == ev["hi"]
    assert np.array_equal(got[certain], ev["grid"][certain])


def test_every_batch_plan_gives_the_default_results(lib):
    import torch

    from paper_2502_06337_gb300 import binding as B

    specs = synth.batch_specs(48, seed=43)
    batch = []
    for s in specs:
        pb = synth.make_problem(s["n"], s["inlier_fracs"], s["sigma"], seed=s["seed"])
        batch.append((torch.from_numpy(pb.P).cuda(), torch.from_numpy(pb.Q).cuda(),
                      B.make_params(grid=0, angle_bins=360, tau=synth.default_tau(s["sigma"]))))
    mean_n = sum(s["n"] for s in specs) // len(specs)
    ref, grids = B.estimate_batch(batch)
    for kn in BATCH:
        B.set_tuned_plan(mean_n, kn, batched=True)
        res, g2 = B.estimate_batch(batch)
        assert np.array_equal(g2, grids)
        for a, b in zip(res, ref):
            _same(a, b)
    B.autotune_reset()
    win = B.autotune_batch(batch, reps=2)
    assert _knob_view(win) in BATCH and 0 < win["ms_tuned"] <= win["ms_default"]
    found, used = B.tuned_plan(mean_n, batched=True)
    assert found and _knob_view(used) == _knob_view(win)
    res, _ = B.estimate_batch(batch)
    for a, b in zip(res, ref):
        _same(a, b)
