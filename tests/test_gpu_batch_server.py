"""The batched and served forms against the plain solve and the FP64 oracle (gpu).

A batch of uneven instances solved in one launch sequence must give, per instance, the same
integer results (cells, bins, counts, sets) as solving that instance alone, and FP64
rotations equal to rounding; the served form must give every request the result it has
alone, whatever else is in flight."""
import numpy as np
import pytest

import oracle
from paper_2502_06337_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu

INT_KEYS = ("cell", "bin", "axis_votes", "angle_votes", "n_vote_set", "n_inliers", "n_degenerate")


def _same(a, b, tol=1e-12):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        for key in INT_KEYS:
            assert x[key] == y[key], (key, x[key], y[key])
        assert parity.rot_diff(x["R"], y["R"]) <= tol
        assert parity.rot_diff(x["R_init"], y["R_init"]) <= tol


def _instances():
    """Uneven instances: sizes from 1 to 60k, outlier rates 30-95 %, one with three
    rotations, one whose pairs are all degenerate (no axis), fixed and autotuned grids."""
    specs = [
        dict(n=700, fr=(0.5,), sigma=0.01, seed=11, grid=128, k=1),
        dict(n=4099, fr=(0.3,), sigma=0.005, seed=12, grid=0, k=1),
        dict(n=60000, fr=(0.05,), sigma=0.01, seed=13, grid=0, k=1),
        dict(n=20000, fr=(0.2, 0.2, 0.2), sigma=0.01, seed=14, grid=256, k=3),
        dict(n=1, fr=(1.0,), sigma=0.0, seed=15, grid=64, k=1),
        dict(n=300, fr=(0.7,), sigma=0.02, seed=16, grid=16, k=2),
        dict(n=3000, fr=(0.4,), sigma=0.01, seed=18, grid=1024, k=1),
    ]
    out = []
    for s in specs:
        pb = synth.make_problem(s["n"], s["fr"], s["sigma"], seed=s["seed"])
        out.append((pb, s))
    # all pairs degenerate: p = q
    P = synth.make_problem(50, (0.0,), 0.0, seed=17).P
    out.append((synth.Problem(P=P, Q=P.copy(), rotations=[], truth=np.full(50, -1), sigma=0.0,
                              seed=17), dict(n=50, grid=32, k=1)))
    return out


def _params(B, s, tau=0.05):
    return B.make_params(grid=s["grid"], angle_bins=360, k=s["k"], nms_deg=2.0, tau=tau)


def test_batch_matches_single_solves(lib):
    import torch

    from paper_2502_06337_gb300 import binding as B

    inst = _instances()
    dev = [(torch.from_numpy(pb.P).cuda(), torch.from_numpy(pb.Q).cuda()) for pb, _ in inst]
    batch = [(P, Q, _params(B, s)) for (P, Q), (_, s) in zip(dev, inst)]
    res, grids = B.estimate_batch(batch)
    for i, ((P, Q), (pb, s)) in enumerate(zip(dev, inst)):
        if s["grid"]:
            assert grids[i] == s["grid"]
        else:
            assert grids[i] == lib.sprot_autotune_grid(pb.n)
        prm = B.make_params(grid=grids[i], angle_bins=360, k=s["k"], nms_deg=2.0, tau=0.05)
        alone = B.estimate_rotations(P, Q, prm, allow_noaxis=True)
        _same(res[i], alone)
    assert res[-1] == []  # the all-degenerate instance finds no axis and does not disturb the rest


def test_batch_small_instances_match_oracle(lib):
    """End to end against the oracle's solve on the small instances of the batch (same grid):
    same cells and bins and rotations within the estimator's 1e-5 rad."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    inst = [x for x in _instances() if x[1]["n"] in (700, 300, 1)]
    batch = [(torch.from_numpy(pb.P).cuda(), torch.from_numpy(pb.Q).cuda(), _params(B, s))
             for pb, s in inst]
    res, grids = B.estimate_batch(batch)
    for (pb, s), r, G in zip(inst, res, grids):
        want = oracle.solve(pb.P, pb.Q, G, 360, k=s["k"], nms_deg=2.0, tau=0.05)
        assert [x["cell"] for x in r] == [(row, col) for row, col, _ in want["peaks"]]
        P64, Q64 = pb.P.astype(np.float64), pb.Q.astype(np.float64)
        for a, x in enumerate(r):
            assert x["bin"] == want["rotations"][a]["bin"]
            sel = want["labels"] == a
            assert x["n_inliers"] == int(sel.sum())
            M = Q64[sel].T @ P64[sel]
            sv = np.linalg.svd(M, compute_uv=False)
            if sel.any() and sv[1] > 1e-6 * sv[0]:
                assert parity.rot_diff(x["R"], want["rotations"][a]["R"]) < parity.E2E_ROT_TOL
            else:
                # one pair or collinear pairs: every maximiser of tr(R^T M) is correct
                R = x["R"]
                assert parity.rot_diff(R @ R.T, np.eye(3)) < 1e-12 and abs(np.linalg.det(R) - 1) < 1e-12
                best = np.trace(want["rotations"][a]["R"].T @ M)
                assert abs(np.trace(R.T @ M) - best) <= 1e-9 * max(1.0, sv[0])


def test_server_results_equal_alone(lib):
    """Requests of different sizes and rotation counts submitted together: each result is
    the one the request gets alone (same integers, FP64 rotations equal to rounding)."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    inst = [x for x in _instances() if x[1]["n"] > 1]
    alone = []
    for pb, s in inst:
        P = torch.from_numpy(pb.P).cuda()
        Q = torch.from_numpy(pb.Q).cuda()
        alone.append(B.estimate_rotations(P, Q, _params(B, s), allow_noaxis=True))
    with B.Server(2 << 30, max_batch=8) as srv:
        for rep in range(3):
            tickets = [srv.submit(pb.P, pb.Q, _params(B, s)) for pb, s in inst]
            got = [srv.wait(t) for t in tickets]
            for (pb, s), g, a in zip(inst, got, alone):
                if a:
                    assert g["status"] == 0
                else:
                    assert g["status"] == B.E_NOAXIS
                _same(g["rotations"], a)
                assert g["t_submit_ms"] <= g["t_admit_ms"] <= g["t_done_ms"]


def test_server_admission_and_invalid_requests(lib):
    from paper_2502_06337_gb300 import binding as B

    pb = synth.make_problem(100_000, (0.2,), 0.01, seed=21)
    with B.Server(1 << 20, max_batch=4) as srv:  # 1 MB budget: the request can never fit
        st, _ = srv.try_submit(pb.P, pb.Q, B.make_params(grid=256, angle_bins=360))
        assert st == B.E_NOMEM
        st, _ = srv.try_submit(pb.P, pb.Q, B.make_params(grid=24, angle_bins=360))  # not a power of two
        assert st == B.E_INVAL
        small = synth.make_problem(200, (0.5,), 0.01, seed=22)
        t = srv.submit(small.P, small.Q, B.make_params(grid=16, angle_bins=90))
        r = srv.wait(t)
        assert r["status"] == 0 and len(r["rotations"]) == 1
        with pytest.raises(B.SprotError) as e:
            srv.wait(t + 1000)  # no such ticket
        assert e.value.status == B.E_INVAL


def test_graph_replay_matches_direct_solves(lib):
    """Two problems of the same shape solved alternately (the shape is captured as a CUDA graph
    on its second call and replayed after): every result equals the direct solve of the same
    problem (the debug-export path, which never uses graphs)."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    probs = [synth.make_problem(30000, (0.2,), 0.01, seed=s) for s in (31, 32)]
    dev = [(torch.from_numpy(p.P).cuda(), torch.from_numpy(p.Q).cuda()) for p in probs]
    prm = B.make_params(grid=256, angle_bins=360, tau=0.05)
    direct = []
    for P, Q in dev:
        dbg = dict(grid=torch.zeros(256 * 256, dtype=torch.int32, device="cuda"))
        direct.append(B.estimate_rotations(P, Q, prm, debug=dbg))
    for rep in range(3):
        for (P, Q), want in zip(dev, direct):
            _same(B.estimate_rotations(P, Q, prm), want, tol=0.0)
    # a batch shape repeated: the graph replays with new tables
    batch = [(P, Q, prm) for P, Q in dev]
    first, _ = B.estimate_batch(batch)
    for rep in range(2):
        again, _ = B.estimate_batch(batch[::-1])
        _same(again[0], first[1], tol=0.0)
        _same(again[1], first[0], tol=0.0)


def test_concurrent_calls_on_separate_streams(lib):
    """Four host threads, each on its own CUDA stream, solve different problems repeatedly
    (the workspaces, graph caches and launch counters are shared library state): every result
    equals the same problem solved alone on the default stream."""
    import threading

    import torch

    from paper_2502_06337_gb300 import binding as B

    probs = [synth.make_problem(n, (0.2,), 0.01, seed=70 + t) for t, n in enumerate((20000, 50000, 3000, 120000))]
    prm = B.make_params(grid=256, angle_bins=360, tau=0.05)
    dev = [(torch.from_numpy(p.P).cuda(), torch.from_numpy(p.Q).cuda()) for p in probs]
    want = [B.estimate_rotation(P, Q, prm) for P, Q in dev]
    errors, got = [], [[] for _ in dev]

    def worker(t):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(6):  # direct, captured, then replayed graphs on this stream
                    got[t].append(B.estimate_rotation(dev[t][0], dev[t][1], prm))  # on s, the thread's current stream
        except Exception as e:  # reported after the join
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(len(dev))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for t in range(len(dev)):
        assert len(got[t]) == 6
        for r in got[t]:
            _same([r], [want[t]], tol=0.0)


def test_server_budget_admits_one_request_at_a_time(lib):
    """Six requests of n = 20,000 at G = 128 under a budget of 1.5 times the bytes the admission
    counts for one of them: each fits alone but no two fit together, so the server must queue
    them, admit one at a time as memory frees up, and still give every request its result
    alone."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    probs = [synth.make_problem(20000, (0.3,), 0.01, seed=80 + i) for i in range(6)]
    prm = B.make_params(grid=128, angle_bins=360, tau=0.05)
    alone = [B.estimate_rotation(torch.from_numpy(p.P).cuda(), torch.from_numpy(p.Q).cuda(), prm) for p in probs]
    with B.Server(1 << 40, max_batch=8) as probe:
        one = probe.request_bytes(probs[0].P, probs[0].Q, prm)
    assert one > 20000 * 24
    with B.Server(one * 3 // 2, max_batch=8) as srv:
        tickets = [srv.submit(p.P, p.Q, prm) for p in probs]
        got = [srv.wait(t) for t in tickets]
    spans = []
    for g, a in zip(got, alone):
        assert g["status"] == 0
        _same(g["rotations"], [a])
        spans.append((g["t_admit_ms"], g["t_done_ms"]))
    spans.sort()
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 0.05, (a0, d0, a1, d1)  # admitted only after the previous one finished


def test_batch_with_a_headline_instance_and_labels(lib):
    """A batch holding the n = 10^6 headline problem beside a 3-rotation instance and two small
    ones, with per-instance label outputs: every instance's rotations and labels equal those of
    its solve alone."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    cfg = synth.HEADLINE
    specs = [(synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0),
              B.make_params(grid=512, angle_bins=720, tau=synth.default_tau(cfg["sigma"]))),
             (synth.make_problem(30000, (0.2, 0.2, 0.2), 0.01, seed=90),
              B.make_params(grid=256, angle_bins=360, k=3, nms_deg=2.0, tau=0.05)),
             (synth.make_problem(4000, (0.5,), 0.01, seed=91), B.make_params(grid=0, tau=0.05)),
             (synth.make_problem(150, (0.6,), 0.01, seed=92), B.make_params(grid=64, tau=0.05))]
    dev = [(torch.from_numpy(p.P).cuda(), torch.from_numpy(p.Q).cuda()) for p, _ in specs]
    labs = [torch.full((p.n,), -7, dtype=torch.int32, device="cuda") for p, _ in specs]
    res, grids = B.estimate_batch([(P, Q, prm, L) for (P, Q), (_, prm), L in zip(dev, specs, labs)])
    for i, ((P, Q), (p, prm)) in enumerate(zip(dev, specs)):
        alone_prm = B.make_params(grid=int(grids[i]), angle_bins=prm.angle_bins, k=prm.k, nms_deg=prm.nms_deg,
                                  tau=prm.tau)
        lab_alone = torch.full((p.n,), -7, dtype=torch.int32, device="cuda")
        alone = B.estimate_rotations(P, Q, alone_prm, labels=lab_alone)
        _same(res[i], alone)
        assert torch.equal(labs[i], lab_alone)


def test_server_cycles_release_device_memory(lib):
    """Creating, using and destroying servers repeatedly does not accumulate device memory:
    each worker's workspace and input arena are freed with its stream."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    prob = synth.make_problem(200_000, (0.2,), 0.01, seed=95)
    prm = B.make_params(grid=0, tau=0.05)

    def cycle():
        with B.Server(4 << 30, max_batch=8) as srv:
            tickets = [srv.submit(prob.P, prob.Q, prm) for _ in range(24)]
            assert all(srv.wait(t)["status"] == 0 for t in tickets)

    cycle()  # the first cycle loads modules and grows the memory pools
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        cycle()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (256 << 20), f"{(free0 - free1) / 2**20:.0f} MiB not returned"


def test_release_stream_workspace_returns_memory(lib):
    """Solving on short-lived streams and releasing each stream's workspace before the stream
    goes (sprot_release_stream_workspace) keeps device memory flat."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    cfg = synth.HEADLINE
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=96)
    P, Q = torch.from_numpy(prob.P).cuda(), torch.from_numpy(prob.Q).cuda()
    prm = B.make_params(grid=512, angle_bins=720, tau=synth.default_tau(cfg["sigma"]))
    want = B.estimate_rotation(P, Q, prm)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(6):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            got = B.estimate_rotation(P, Q, prm)  # a workspace for s (about 35 MB at this size)
        _same([got], [want], tol=0.0)
        B.release_stream_workspace(s.cuda_stream)
        del s
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (64 << 20), f"{(free0 - free1) / 2**20:.0f} MiB not returned"
    B.release_stream_workspace(torch.cuda.current_stream().cuda_stream)  # no-op-safe on a used stream too


def test_packed_batch_matches_list_batch(lib):
    """The packed form (all pairs back to back, offsets, a params record array, one labels
    tensor) gives every instance the results and labels of the list form."""
    import torch

    from paper_2502_06337_gb300 import binding as B

    inst = [x for x in _instances() if x[1]["n"] > 1]
    P = torch.from_numpy(np.concatenate([pb.P for pb, _ in inst])).cuda()
    Q = torch.from_numpy(np.concatenate([pb.Q for pb, _ in inst])).cuda()
    off = np.concatenate([[0], np.cumsum([pb.n for pb, _ in inst])])
    arr = B.params_array(len(inst), grid=[s["grid"] for _, s in inst], angle_bins=360, k=[s["k"] for _, s in inst],
                         nms_deg=2.0, tau=0.05)
    lab = torch.full((int(off[-1]),), -7, dtype=torch.int32, device="cuda")
    res, grids = B.estimate_batch_packed(P, Q, off, arr, labels=lab)
    lst = [(P[off[i]:off[i + 1]], Q[off[i]:off[i + 1]], _params(B, s),
            torch.full((pb.n,), -7, dtype=torch.int32, device="cuda")) for i, (pb, s) in enumerate(inst)]
    ref, grids_l = B.estimate_batch(lst)
    assert np.array_equal(grids, grids_l)
    for i in range(len(inst)):
        _same(res[i], ref[i], tol=0.0)
        assert torch.equal(lab[off[i]:off[i + 1]], lst[i][3])
