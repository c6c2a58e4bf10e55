"""Writes the oracle-derived regression fixtures of this folder. Calls only ``oracle`` and
the seeded input generator; never the CUDA library.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2502_06337_gb300 import synth  # noqa: E402


def small_seed0():
    cfg = synth.SMALL
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    tau = synth.default_tau(cfg["sigma"])
    out = oracle.solve(prob.P, prob.Q, cfg["grid"], cfg["angle_bins"], tau=tau)
    rot = out["rotations"][0]
    return dict(
        source="oracle.solve on synth.make_problem(1000, (0.5,), 0.01, seed=0), G=256, J=360",
        tau=tau,
        cell=list(rot["cell"]),
        axis_votes=int(rot["axis_votes"]),
        bin=int(rot["bin"]),
        n_inliers=int((out["labels"] >= 0).sum()),
        R=rot["R"].tolist(),
    )


if __name__ == "__main__":
    with open(os.path.join(HERE, "small_seed0.json"), "w") as f:
        json.dump(small_seed0(), f, indent=1)
    print("wrote small_seed0.json")
