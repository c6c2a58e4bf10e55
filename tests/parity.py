"""Stage-by-stage comparison of the CUDA path with the FP64 oracle (helpers for the gpu
tests). Integer results must equal the oracle's wherever the oracle did not flag the decision
as within the boundary band, and lie within the oracle's bounds elsewhere; FP64 rotations
must agree with the oracle's least squares on the same sets to 1e-9 rad (the estimator's
stated tolerance is 1e-5 rad)."""
from __future__ import annotations

import numpy as np

import oracle

ROT_TOL = 1e-9      # FP64 refinement, same inputs, different summation order (max |dR|)
E2E_ROT_TOL = 1e-5  # end to end against the oracle's own solve (radians, Eq. 16)


def rot_diff(Ra, Rb) -> float:
    """max |Ra - Rb| over the entries: about the angle between them in radians for small
    angles, and well conditioned there (Eq. 16's arccos cannot resolve angles below ~1.5e-8
    rad in float64, its argument being within rounding of 1)."""
    return float(np.max(np.abs(np.asarray(Ra) - np.asarray(Rb))))


def check_lsq(P_sel, Q_sel, R_gpu, R_fallback):
    """The GPU least-squares rotation over a set against the oracle's Kabsch. When
    M = sum q p^T has two well separated non-zero singular values the optimum is unique and
    the matrices are compared; otherwise (one pair, collinear pairs) every maximiser of
    tr(R^T M) is correct, so the objective value and the validity of R are compared."""
    R_gpu = np.asarray(R_gpu)
    if len(P_sel) == 0:
        assert rot_diff(R_fallback, R_gpu) < ROT_TOL
        return
    M = np.asarray(Q_sel, dtype=np.float64).T @ np.asarray(P_sel, dtype=np.float64)
    s = np.linalg.svd(M, compute_uv=False)
    R_ref = oracle.kabsch(P_sel, Q_sel)
    if s[1] > 1e-6 * s[0]:
        assert rot_diff(R_ref, R_gpu) < ROT_TOL, rot_diff(R_ref, R_gpu)
    else:
        assert rot_diff(R_gpu @ R_gpu.T, np.eye(3)) < 1e-12 and abs(np.linalg.det(R_gpu) - 1) < 1e-12
        best = np.trace(R_ref.T @ M)
        assert abs(np.trace(R_gpu.T @ M) - best) <= 1e-12 * max(1.0, s[0])


def run_gpu(P, Q, G, J, k=1, nms=2.0, w=1, window=1, tau=0.05, host=False, subcell=False):
    """The CUDA solve with every intermediate exported. Returns a dict of numpy arrays."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    n = P.shape[0]
    dev = torch.device("cuda")
    Pt = torch.from_numpy(np.ascontiguousarray(P)).to(dev)
    Qt = torch.from_numpy(np.ascontiguousarray(Q)).to(dev)
    dbg = dict(
        grid=torch.zeros(G * G, dtype=torch.int32, device=dev),
        hist=torch.zeros(k * J, dtype=torch.int32, device=dev),
        bins=torch.zeros(k * n, dtype=torch.int16, device=dev),
        vote_set=torch.zeros(k * n, dtype=torch.uint8, device=dev),
    )
    labels = torch.zeros(n, dtype=torch.int32, device=dev)
    prm = B.make_params(grid=G, angle_bins=J, k=k, nms_deg=nms, gate_window=w, angle_window=window, tau=tau,
                        flags=B.SUBCELL_AXIS if subcell else 0)
    rots = B.estimate_rotations(Pt, Qt, prm, labels=labels, debug=dbg, allow_noaxis=True)
    torch.cuda.synchronize()
    u32 = lambda t: t.cpu().numpy().view(np.uint32).astype(np.int64)
    return dict(
        rots=rots,
        grid=u32(dbg["grid"]).reshape(G, G),
        hist=u32(dbg["hist"]).reshape(k, J),
        bins=dbg["bins"].cpu().numpy().reshape(k, n).astype(np.int64),
        vote_set=dbg["vote_set"].cpu().numpy().reshape(k, n).astype(bool),
        labels=labels.cpu().numpy(),
    )


def check_grid(gpu_grid, av, what=""):
    """lo <= gpu <= hi everywhere; equal to the oracle where no decision was flagged."""
    lo, hi, grid = av["lo"], av["hi"], av["grid"]
    bad_bounds = int(((gpu_grid < lo) | (gpu_grid > hi)).sum())
    certain = lo == hi
    bad_exact = int(((gpu_grid != grid) & certain).sum())
    assert bad_bounds == 0 and bad_exact == 0, (
        f"{what}: {bad_bounds} cells outside the oracle bounds, {bad_exact} unflagged cells differ")
    return int((~certain).sum())


def check_solve(P, Q, g, G, J, k=1, nms=2.0, w=1, window=1, tau=0.05, av=None, subcell=False):
    """Every stage of one GPU solve ``g`` (from run_gpu) against the oracle. ``av`` may hold a
    precomputed oracle axis vote; ``subcell``: the solve used the sub-cell axis. Returns a dict
    of flagged counts."""
    P = np.asarray(P, dtype=np.float32)
    Q = np.asarray(Q, dtype=np.float32)
    report = {}
    if av is not None:
        report["flagged_cells"] = check_grid(g["grid"], av, "grid")
    # peaks: the oracle's greedy top-k on the GPU grid
    peaks = oracle.top_k_cells(g["grid"], k, nms)
    assert [(r["cell"][0], r["cell"][1], r["axis_votes"]) for r in g["rots"]] == peaks
    R1s = []
    for a, rot in enumerate(g["rots"]):
        row, col = rot["cell"]
        # sub-cell offsets: exact integer arithmetic and one quotient on both sides
        off = oracle.subcell_offset(g["grid"], row, col)
        assert rot["cell_offset"] == off, (rot["cell_offset"], off)
        r = oracle.subcell_axis(G, row, col, *off) if subcell else oracle.cell_axis(G, row, col)
        gate, gflag = oracle.window_gate(P, Q, G, row, col, w)
        av_ = oracle.angle_vote(P, Q, r, gate, gflag, J)
        hist = g["hist"][a]
        assert np.all(hist >= av_["lo"]) and np.all(hist <= av_["hi"]), "angle histogram outside bounds"
        certain = av_["member_lo"] & ~av_["bin_flag"]
        assert np.array_equal(g["bins"][a][certain], av_["bin"][certain]), "angle bins differ"
        assert np.all(g["bins"][a][~av_["member_hi"]] == -1), "pair voted that cannot vote"
        b, th = oracle.angle_peak(hist)
        assert rot["bin"] == b and rot["angle_votes"] == int(hist[b])
        # axis and R_vote are exact functions of (cell, bin)
        axis, theta = (r, th) if th >= 0 else (-r, -th)
        assert np.allclose(rot["axis"], axis, atol=4e-16 * G) and abs(rot["theta"] - theta) < 1e-14
        assert np.allclose(rot["R_vote"], oracle.rodrigues(axis, theta), atol=1e-14)
        V, V_lo, V_hi = oracle.vote_set(av_, b, J, window)
        gv = g["vote_set"][a]
        assert np.all(gv[V_lo]) and not np.any(gv & ~V_hi), "vote set outside bounds"
        assert rot["n_vote_set"] == int(gv.sum())
        check_lsq(P[gv], Q[gv], rot["R_init"], rot["R_vote"])
        R1s.append(rot["R_init"])
        report.setdefault("flagged_pairs", 0)
        report["flagged_pairs"] += int((av_["member_hi"] & ~(av_["member_lo"] & ~av_["bin_flag"])).sum())
    labels, lflag = oracle.assign_labels(P, Q, R1s, tau)
    assert np.array_equal(g["labels"][~lflag], labels[~lflag]), "labels differ"
    report["flagged_labels"] = int(lflag.sum())
    for a, rot in enumerate(g["rots"]):
        sel = g["labels"] == a
        assert rot["n_inliers"] == int(sel.sum())
        check_lsq(P[sel], Q[sel], rot["R"], rot["R_init"])
    return report
