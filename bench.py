"""Benchmark of the stereographic-projection rotation vote on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sprot|reference] [--no-extras]

A step is one whole solve of the headline workload -- n = 10^6 correspondences, 90 %
outliers, inlier noise 0.01, 512 x 512 axis grid, 720 angle bins -- through the C ABI:
axis vote, peak, angle vote, Rodrigues, FP64 refinement and labels. The JSON line reports
Mcorr/s = n / (device time per step) with inputs resident in HBM (``value``), the same
through host buffers with the copies inside the timed region (``e2e``), the roofline of the
axis-vote kernel, the FP64 oracle timed on the host cores on a bounded sample
(``cpu_baseline``), and, unless --no-extras, the batched (4096 instances) and served
(Poisson 2000 req/s) forms.

With N > 1 (torchrun, one process per GPU) every rank solves its own replica of the
workload: the vote does not need any exchange, so there is no collective on the data path.
``--impl reference`` times the FP64 oracle (the only reference there is) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mcorr/s axis+angle vote (n=1e6, 90% outl.); served solves/s, p50/p99 ms"
WORKLOAD = "single rotation, n=1e6, 90% outliers, sigma=0.01, 512x512 grid, 720 angle bins"
UNIT = "Mcorr/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB of L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sprot", choices=["sprot", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default="all",
                    help="comma-separated extras to run (multi_rotation, paper_recipe, ls_axis, "
                         "sampled_vote, eps_vote, batched, served) or 'all'")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the oracle CPU baseline (profiling runs)")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="correspondences of the oracle baseline sample (default 2000 per host core)")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------
# distributed helpers (replicas only)
# ---------------------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Maximum of a per-rank scalar (the slowest replica sets the job time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# the headline workload on the GPU
# ---------------------------------------------------------------------------------------

def vote_profile():
    """The committed ncu record of the axis-vote kernel (DRAM bytes and warp instructions per
    launch), or {} when the kernel source has changed since the counters were taken."""
    prof = os.path.join(ROOT, "profiles", "axis_vote_traffic.json")
    src = os.path.join(ROOT, "paper_2502_06337_gb300", "csrc", "vote_runs.cu")
    try:
        rec = json.load(open(prof))
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return {}
    return rec if rec.get("kernel_source_sha256") == digest else {}


def headline_problem(seed):
    from paper_2502_06337_gb300 import synth

    cfg = synth.HEADLINE
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=seed)
    return prob, cfg


def run_sprot(args):
    import torch

    from paper_2502_06337_gb300 import binding as B
    from paper_2502_06337_gb300 import build as Bd
    from paper_2502_06337_gb300 import synth

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    if not os.path.exists(B.LIB_PATH):
        Bd.build()
    B.load()
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    prob, cfg = headline_problem(seed=rank)
    n = prob.n
    G, J, tau = cfg["grid"], cfg["angle_bins"], synth.default_tau(cfg["sigma"])
    prm = B.make_params(grid=G, angle_bins=J, tau=tau)
    P = torch.from_numpy(prob.P).to(dev)
    Q = torch.from_numpy(prob.Q).to(dev)
    mask = torch.zeros(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        return B.estimate_rotation(P, Q, prm, mask=mask)

    for _ in range(max(3, args.warmup)):
        rot = step()
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs) ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    launches0 = B.launch_count()
    B.kernel_timing(True)
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))  # L2 flush between timed steps (outside the events)
            ev[i][0].record(st)
            rot = step()
            ev[i][1].record(st)
        torch.cuda.synchronize()
    vote_ms, vote_launches = B.kernel_timing_read()
    B.kernel_timing(False)
    launches = B.launch_count() - launches0
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1e3
    t_job = max_over_ranks(t_local, world, dev)
    value = world * n * args.steps / t_job / 1e6
    clocks = clk.summary()

    # ---- end to end through host buffers (copies inside the timed region) ----
    Ph = torch.from_numpy(prob.P).pin_memory()
    Qh = torch.from_numpy(prob.Q).pin_memory()
    mh = torch.zeros(n, dtype=torch.uint8).pin_memory()
    prm_h = B.make_params(grid=G, angle_bins=J, tau=tau, flags=B.HOST_PTRS)
    Pn, Qn, mn = Ph.numpy(), Qh.numpy(), mh.numpy()
    for _ in range(2):
        B.estimate_rotation(Pn, Qn, prm_h, mask=mn)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rot_h = B.estimate_rotation(Pn, Qn, prm_h, mask=mn)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    t_e2e = max_over_ranks(sum(e2e_ms) / 1e3, world, dev)
    e2e = {"value": world * n * args.steps / t_e2e / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(prob.P.nbytes + prob.Q.nbytes),
           "d2h_bytes_per_step": int(n + 280),
           "api": "sprot_estimate_rotation(SPROT_HOST_PTRS)"}
    assert rot_h["cell"] == rot["cell"] and np.array_equal(rot_h["R"], rot["R"])

    # ---- roofline of the axis-vote kernel ----
    grid = torch.zeros(G * G, dtype=torch.int32, device=dev)
    B.axis_vote(P, Q, G, grid)
    torch.cuda.synchronize()
    increments = int(grid.cpu().numpy().view(np.uint32).astype(np.int64).sum())
    atomic_peak = B.probe_smem_atomic_rate(4096)
    vote_s = vote_ms / 1e3 / max(1, vote_launches)
    achieved = increments / vote_s
    roofline = {
        "bound": "alu",
        "resource": "shared-memory atomic unit (the rate of one red.shared.add.u32 per voted cell)",
        "kernel": "k_axis_vote_runs",
        "achieved": achieved / 1e9,
        "peak": atomic_peak / 1e9,
        "unit": "Gatom/s",
        "frac": achieved / atomic_peak,
        "peak_source": "measured in this run by sprot_probe_smem_atomic_rate (conflict-free shared atomics on every SM)",
        "algorithmic_per_launch": increments,
        "kernel_ms": vote_s * 1e3,
        "kernel_share_of_step": vote_s * 1e3 / (sum(step_ms) / len(step_ms)),
        "traffic": None,
    }
    rec = vote_profile()
    roofline["traffic"] = rec.get("dram_bytes_per_launch")
    # instruction issue, the kernel's binding limit: warp instructions per launch (committed
    # capture of the same source) over the live kernel time, against 4 issue slots per SM per
    # cycle at the SM clock sampled during the timed region
    if rec.get("warp_instructions_per_launch") and clocks.get("sm_mhz"):
        slots = rec["grid_ctas"] * 4 * clocks["sm_mhz"] * 1e6
        roofline["issue"] = {"achieved_warp_inst_per_s": rec["warp_instructions_per_launch"] / vote_s,
                             "peak_warp_inst_per_s": slots, "unit": "warp instructions/s",
                             "frac": rec["warp_instructions_per_launch"] / vote_s / slots,
                             "note": "SMs the grid occupies x 4 schedulers x measured SM clock"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_job * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "dtype_detail": "f32 geometry, u32 vote counts, f64 least-squares refinement",
        "data": "synthetic (seeded; uniform cube points, uniform random rotation)",
        "config": {"workload": WORKLOAD,
                   "n": n, "grid": G, "angle_bins": J, "tau": tau, "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (512 MB write outside the timed events)"},
        "result": {"cell": rot["cell"], "bin": rot["bin"], "axis_votes": rot["axis_votes"],
                   "n_inliers": rot["n_inliers"],
                   "rot_err_deg_vs_truth": math.degrees(_rot_err(prob.rotations[0], rot["R"]))},
        "e2e": e2e, "roofline": roofline, "clocks": clocks,
        "gpu_launches": int(launches), "step_ms_min": min(step_ms), "step_ms_median": float(np.median(step_ms)),
    }
    if rank == 0:
        if not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(prob, G, J, tau, args.cpu_sample)
        if not args.no_extras:
            extras = [("multi_rotation", lambda: run_multi(B, dev)),
                      ("paper_recipe", lambda: run_paper_recipe(B, dev)),
                      ("ls_axis", lambda: run_ls_axis(B, dev)),
                      ("sampled_vote", lambda: run_sampled(B, P, Q, G)),
                      ("eps_vote", lambda: run_eps(B, P, Q, G)),
                      ("batched", lambda: run_batched(B, dev)),
                      ("served", lambda: run_served(B))]
            wanted = None if args.extras == "all" else set(args.extras.split(","))
            for name, fn in extras:
                if wanted is not None and name not in wanted:
                    continue
                try:
                    out[name] = fn()
                except Exception as e:  # report, never hide
                    out[name] = {"error": repr(e)}
        print(json.dumps(out), flush=True)
    barrier(world)
    if world > 1:
        dist.destroy_process_group()


def _rot_err(Ra, Rb):
    c = 0.5 * (np.trace(np.asarray(Ra).T @ np.asarray(Rb)) - 1.0)
    return float(np.arccos(np.clip(c, -1.0, 1.0)))


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------------------

def _oracle_grid(args):
    """Pool task: the oracle's accumulator of one chunk of pairs (grids of disjoint chunks
    add up to the grid of their union)."""
    import oracle

    P, Q, G = args
    return oracle.axis_vote(P, Q, G)["grid"]


class OraclePool:
    """The FP64 oracle on every host core: a spawn process pool (started without fork, so it
    is safe after CUDA is initialised) computes the accumulator over chunks of the pairs; the
    summed grid then goes through the oracle's later stages (peak, angle vote, refinement) in
    this process."""

    def __init__(self):
        import multiprocessing as mp

        self.cores = os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")  # one thread per process
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        z = np.zeros((1, 3), dtype=np.float32)
        self.pool.map(_oracle_grid, [(z, z, 16)] * self.cores)  # workers up and importing done

    def solve(self, P, Q, G, J, tau):
        import oracle

        parts = np.array_split(np.arange(len(P)), self.cores)
        grids = self.pool.map(_oracle_grid, [(P[ix], Q[ix], G) for ix in parts if len(ix)])
        return oracle.solve(P, Q, G, J, tau=tau, grid=np.sum(grids, axis=0))

    def time(self, P, Q, G, J, tau):
        t0 = time.perf_counter()
        self.solve(P, Q, G, J, tau)
        return time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_baseline(prob, G, J, tau, n_s):
    """The oracle on all host cores on the first n_s pairs of the workload, plus one thread on
    the small workload (n = 1000, 256^2, 360 bins)."""
    import oracle
    from paper_2502_06337_gb300 import synth

    pool = OraclePool()
    try:
        n_s = n_s or 2000 * pool.cores
        t = pool.time(prob.P[:n_s], prob.Q[:n_s], G, J, tau)
    finally:
        pool.close()
    cfg = synth.SMALL
    small = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    t0 = time.perf_counter()
    oracle.solve(small.P, small.Q, cfg["grid"], cfg["angle_bins"], tau=synth.default_tau(cfg["sigma"]))
    t1 = time.perf_counter() - t0
    return {"value": n_s / t / 1e6, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"first {n_s} correspondences of the n=1e6 workload (same G={G}, J={J}), "
                      f"{t:.1f} s wall on {pool.cores} processes (accumulator split by pairs, later "
                      f"stages in one process); numpy float64",
            "one_thread_small": {"workload": f"n={cfg['n']}, {cfg['grid']}x{cfg['grid']}, {cfg['angle_bins']} bins",
                                 "s": t1, "Mcorr_per_s": cfg["n"] / t1 / 1e6}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2502_06337_gb300 import synth

    prob, cfg = headline_problem(seed=0)
    G, J, tau = cfg["grid"], cfg["angle_bins"], synth.default_tau(cfg["sigma"])
    pool = OraclePool()
    try:
        n_s = 500 * pool.cores
        P, Q = prob.P[:n_s], prob.Q[:n_s]
        for _ in range(max(1, min(args.warmup, 1))):
            pool.time(P, Q, G, J, tau)
        times = [pool.time(P, Q, G, J, tau) for _ in range(args.steps)]
    finally:
        pool.close()
    t = sum(times)
    value = n_s * args.steps / t / 1e6
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD,
                                        "n": prob.n, "grid": G, "angle_bins": J},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": f"each step: FP64 oracle on the first {n_s} correspondences, "
                                   f"accumulator split over {pool.cores} processes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------------------
# batched and served forms
# ---------------------------------------------------------------------------------------

def run_multi(B, dev, reps=10):
    """Three rotations owning 15 % each, 55 % outliers, n = 2e5, 512^2, 720 bins, top 3 with
    2 degree suppression: time per solve (device-resident) and each true rotation's error."""
    import torch

    from paper_2502_06337_gb300 import synth

    cfg = synth.MULTI
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=3)
    P = torch.from_numpy(prob.P).to(dev)
    Q = torch.from_numpy(prob.Q).to(dev)
    prm = B.make_params(grid=cfg["grid"], angle_bins=cfg["angle_bins"], k=cfg["k"], nms_deg=cfg["nms_deg"],
                        tau=synth.default_tau(cfg["sigma"]))
    for _ in range(3):
        rots = B.estimate_rotations(P, Q, prm)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        rots = B.estimate_rotations(P, Q, prm)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    errs = [min(math.degrees(_rot_err(Rg, r["R"])) for r in rots) for Rg in prob.rotations]
    return {"workload": "n=2e5, 3 x 15% inliers, 55% outliers, sigma=0.01, 512x512, 720 bins, k=3, NMS 2 deg",
            "ms": ms, "Mcorr_per_s": prob.n / ms / 1e3, "found": len(rots),
            "rot_err_deg_vs_truth": errs}


def run_paper_recipe(B, dev, reps=10):
    """The paper's own synthetic recipe (Sec. V-A: unit-length points, 90 % outliers, sigma
    0.01, n = 10^6) through the same solve: time per solve (device-resident inputs, L2 warm)
    and the error against the true rotation. The paper reports 0.07 s and 0.01 degrees on an
    RTX 4080 (context, not a target)."""
    import torch

    from paper_2502_06337_gb300 import synth

    prob = synth.make_problem(1_000_000, (0.1,), 0.01, seed=7, unit=True)
    P = torch.from_numpy(prob.P).to(dev)
    Q = torch.from_numpy(prob.Q).to(dev)
    prm = B.make_params(grid=512, angle_bins=720, tau=synth.default_tau(0.01))
    for _ in range(3):
        rot = B.estimate_rotation(P, Q, prm)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        rot = B.estimate_rotation(P, Q, prm)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    return {"workload": "n=1e6 unit-length points, 90% outliers, sigma=0.01 (Sec. V-A), 512x512, 720 bins",
            "ms": ms, "Mcorr_per_s": prob.n / ms / 1e3, "n_inliers": rot["n_inliers"],
            "rot_err_deg_vs_truth": math.degrees(_rot_err(prob.rotations[0], rot["R"])),
            "paper": {"s": 0.07, "rot_err_deg": 0.01, "gpu": "RTX 4080"}}


def run_ls_axis(B, dev, reps=20):
    """The least-squares axis of Eq. 10 (sprot_refine_axis) on the headline pairs labelled by a
    solve: time per call and the angle to the refined rotation's axis."""
    import torch

    from paper_2502_06337_gb300 import synth

    cfg = synth.HEADLINE
    prob = synth.make_problem(cfg["n"], cfg["inlier_fracs"], cfg["sigma"], seed=0)
    P = torch.from_numpy(prob.P).to(dev)
    Q = torch.from_numpy(prob.Q).to(dev)
    labels = torch.empty(prob.n, dtype=torch.int32, device=dev)
    prm = B.make_params(grid=cfg["grid"], angle_bins=cfg["angle_bins"], tau=synth.default_tau(cfg["sigma"]))
    rot = B.estimate_rotations(P, Q, prm, labels=labels)[0]
    for _ in range(3):
        ax = B.refine_axis(P, Q, labels, 0, hint=rot["axis"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        ax = B.refine_axis(P, Q, labels, 0, hint=rot["axis"])
    ms = (time.perf_counter() - t0) * 1e3 / reps
    w, V = np.linalg.eig(rot["R"])
    r = np.real(V[:, np.argmin(np.abs(w - 1.0))])
    ang = math.degrees(math.acos(min(1.0, abs(float(r @ ax["axis"]) / np.linalg.norm(r)))))
    return {"workload": "n=1e6 headline pairs, the solve's inlier labels", "ms_per_call_wall": ms,
            "pairs_used": ax["count"], "deg_to_refined_rotation_axis": ang}


def run_sampled(B, P, Q, G, J=360, reps=5):
    """Algorithm 1's sampled accumulator (J points per circle) on the headline pairs."""
    import torch

    n = P.shape[0]
    grid = torch.zeros(G * G, dtype=torch.int32, device=P.device)
    B.axis_vote_sampled(P, Q, G, J, grid)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        B.axis_vote_sampled(P, Q, G, J, grid)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    votes = int(grid.cpu().numpy().view(np.uint32).astype(np.int64).sum())
    return {"points_per_circle": J, "grid": G, "ms": ms, "Mcorr_per_s": n / ms / 1e3,
            "Gpoints_per_s": n * J / ms / 1e6, "votes": votes, "Gvotes_per_s": votes / ms / 1e6,
            "note": "L2 atomics (red.global.add) into the grid; inputs L2-warm"}


def run_eps(B, P, Q, G, reps=5):
    """The eps-band accumulator of Eq. 9 (sprot_axis_vote_eps: vote and slice reduction into a
    caller grid) on the headline pairs at eps = 0, 0.002 and 0.01."""
    import torch

    n = P.shape[0]
    grid = torch.zeros(G * G, dtype=torch.int32, device=P.device)
    st = torch.cuda.current_stream()
    out = {"workload": f"n={n} headline pairs, {G}^2", "grid": G}
    for eps in (0.0, 0.002, 0.01):
        B.axis_vote_eps(P, Q, G, eps, grid)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            B.axis_vote_eps(P, Q, G, eps, grid)
        b.record(st)
        torch.cuda.synchronize()
        votes = int(grid.cpu().numpy().view(np.uint32).astype(np.int64).sum())
        out[f"eps={eps:g}"] = {"ms_per_call": a.elapsed_time(b) / reps, "votes": votes}
    out["note"] = "each call uploads its work table, votes, reduces and synchronizes its stream"
    return out


def run_batched(B, dev, m=4096):
    """4096 uneven instances in one batched solve (packed: all pairs back to back in one tensor,
    with offsets), with the default plan and with the plan the autotuner picks for the batch's
    class; the same batch through the list form (one tensor pair per instance); and a
    per-instance loop of single solves over all 4096 instances."""
    import torch

    from paper_2502_06337_gb300 import synth

    specs = synth.batch_specs(m, seed=0)
    probs = [synth.make_problem(s["n"], s["inlier_fracs"], s["sigma"], seed=s["seed"]) for s in specs]
    off = np.concatenate([[0], np.cumsum([s["n"] for s in specs])]).astype(np.int64)
    total = int(off[-1])
    P_all = torch.from_numpy(np.concatenate([pb.P for pb in probs])).to(dev)
    Q_all = torch.from_numpy(np.concatenate([pb.Q for pb in probs])).to(dev)
    taus = np.array([synth.default_tau(s["sigma"]) for s in specs])
    prm = B.params_array(m, grid=0, angle_bins=360, tau=taus)
    reps = 3

    def timed(call):
        call()  # warm-up (workspace, graph capture)
        call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = call()
        return (time.perf_counter() - t0) / reps, out

    B.autotune_reset()
    t_batch, (res, grids) = timed(lambda: B.estimate_batch_packed(P_all, Q_all, off, prm))
    views = [(P_all[off[i]:off[i + 1]], Q_all[off[i]:off[i + 1]]) for i in range(m)]
    lst = [(P, Q, B.make_params(grid=0, angle_bins=360, tau=float(taus[i]))) for i, (P, Q) in enumerate(views)]
    t_list, (res_l, _) = timed(lambda: B.estimate_batch(lst))
    knobs = B.autotune_batch_packed(P_all, Q_all, off, prm, reps=2)
    t_tuned, (res_t, _) = timed(lambda: B.estimate_batch_packed(P_all, Q_all, off, prm))
    B.autotune_reset()
    # per-instance loop of the plain single solve on every instance (same params and G)
    for i in range(8):
        B.estimate_rotations(*views[i], B.make_params(grid=int(grids[i]), angle_bins=360, tau=float(taus[i])),
                             allow_noaxis=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loop_res = []
    for i, (P, Q) in enumerate(views):
        p1 = B.make_params(grid=int(grids[i]), angle_bins=360, tau=float(taus[i]))
        loop_res.append(B.estimate_rotations(P, Q, p1, allow_noaxis=True))
    t_loop = time.perf_counter() - t0
    # integer results identical; FP64 rotations equal up to summation order (max |dR|; the
    # arccos of Eq. 16 cannot resolve differences this small)

    def same(ra, rb):
        return all(len(a) == len(b) and all(x["cell"] == y["cell"] and x["bin"] == y["bin"] and
                                            x["n_inliers"] == y["n_inliers"] and
                                            float(np.max(np.abs(x["R"] - y["R"]))) < 1e-9 for x, y in zip(a, b))
                   for a, b in zip(ra, rb))

    errs = [math.degrees(_rot_err(pb.rotations[0], r[0]["R"])) for pb, r in zip(probs, res) if r]
    return {"instances": m, "correspondences": total, "batch_s": t_batch,
            "solves_per_s": m / t_batch, "Mcorr_per_s": total / t_batch / 1e6,
            "form": "packed: one P and one Q tensor, offsets, a params record array",
            "list_form": {"solves_per_s": m / t_list, "batch_s": t_list,
                          "note": "one tensor pair and Params per instance (per-instance Python marshalling)",
                          "same_results": bool(same(res_l, res))},
            "tuned": {"knobs": {k: knobs[k] for k in ("batch_slice", "batch_div")},
                      "solves_per_s": m / t_tuned, "batch_s": t_tuned,
                      "tuner_ms_default": knobs["ms_default"], "tuner_ms_tuned": knobs["ms_tuned"],
                      "same_results_as_untuned": bool(same(res_t, res))},
            "loop_solves_per_s": m / t_loop, "speedup_vs_loop": t_loop / t_batch,
            "loop_instances": m, "same_results_as_loop": bool(same(res, loop_res)),
            "median_rot_err_deg": float(np.median(errs)) if errs else None,
            "frac_rot_err_below_1deg": float(np.mean(np.array(errs) < 1.0)) if errs else None}


def run_served(B, duration_s=3.0, rate_hz=2000.0, pool=48, budget_gb=40, saturated_requests=3000,
               in_flight=256):
    """The continuous-batching server on the served mix (n log-uniform in [1e3, 1e6], 1-3
    rotations; host inputs): (1) Poisson arrivals at rate_hz, latency from submit to done;
    (2) at capacity: a closed loop keeping in_flight requests submitted, its throughput and
    latency; (3) the same request sequence as a loop of plain single solves from host
    inputs (sprot_estimate_rotations_k with HOST_PTRS, one call after another)."""
    from collections import deque

    from paper_2502_06337_gb300 import synth

    m = int(duration_s * rate_hz)
    specs = synth.serve_specs(m, seed=1, rate_hz=rate_hz)
    # a pool of distinct problems drawn from the same distribution, reused by the arrivals
    pool_specs = synth.serve_specs(pool, seed=2, rate_hz=rate_hz)
    probs = []
    for s in pool_specs:
        pb = synth.make_problem(s["n"], s["inlier_fracs"], s["sigma"], seed=s["seed"])
        k = len(s["inlier_fracs"])
        probs.append((pb, B.make_params(grid=0, angle_bins=360, k=k, nms_deg=2.0, tau=synth.default_tau(0.01))))
    rng = np.random.default_rng(3)
    seq = [int(j) for j in rng.integers(0, pool, size=saturated_requests)]
    srv = B.Server(budget_gb << 30, max_batch=256)
    try:
        # warm-up: every pool problem once, all in flight (sizes the workers' arenas and
        # workspaces before timing)
        for t in [srv.submit(pb.P, pb.Q, prm) for pb, prm in probs]:
            srv.wait(t)
        tickets = []
        t0 = time.perf_counter()
        for i, s in enumerate(specs):
            dt = s["t_arrive"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            pb, prm = probs[i % pool]
            tickets.append((srv.submit(pb.P, pb.Q, prm), i % pool))
        results = [(srv.wait(t), j) for t, j in tickets]
        wall = time.perf_counter() - t0
        # closed loop at capacity
        sat = []
        q = deque()
        t1 = time.perf_counter()
        for j in seq:
            if len(q) >= in_flight:
                sat.append(srv.wait(q.popleft()))
            pb, prm = probs[j]
            q.append(srv.submit(pb.P, pb.Q, prm))
        while q:
            sat.append(srv.wait(q.popleft()))
        sat_wall = time.perf_counter() - t1
    finally:
        srv.close()
    # the same sequence as a loop of plain solves from host inputs
    host = []
    for pb, prm in probs:
        p1 = B.make_params(grid=prm.grid, angle_bins=prm.angle_bins, k=prm.k, nms_deg=prm.nms_deg,
                           tau=prm.tau, flags=B.HOST_PTRS)
        host.append((pb.P, pb.Q, p1))
    for P, Q, p1 in host[:8]:
        B.estimate_rotations(P, Q, p1, allow_noaxis=True)
    t2 = time.perf_counter()
    loop = [B.estimate_rotations(*host[j], allow_noaxis=True) for j in seq]
    loop_wall = time.perf_counter() - t2
    # the GPU-bound ceiling: the same sequence from device-resident inputs, solved as batches of
    # in_flight requests with no host copies
    import torch

    dev_probs = [(torch.from_numpy(pb.P).cuda(), torch.from_numpy(pb.Q).cuda(), prm) for pb, prm in probs]
    chunks = [[dev_probs[j] for j in seq[a:a + in_flight]] for a in range(0, len(seq), in_flight)]
    B.estimate_batch(chunks[0])
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    for c in chunks:
        B.estimate_batch(c)
    ceiling_wall = time.perf_counter() - t3
    del dev_probs, chunks
    same = all(len(r["rotations"]) == len(lr) and
               all(tuple(a["cell"]) == tuple(b["cell"]) and a["bin"] == b["bin"] and a["n_inliers"] == b["n_inliers"]
                   for a, b in zip(r["rotations"], lr))
               for r, lr in zip(sat, loop))
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r, _ in results])
    first = min(r["t_submit_ms"] for r, _ in results)
    last = max(r["t_done_ms"] for r, _ in results)
    ok = sum(1 for r, _ in results if r["status"] == 0)
    corr = sum(probs[j][0].n for _, j in results)
    sat_lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in sat])
    sat_corr = sum(probs[j][0].n for j in seq)
    return {"requests": m, "completed_ok": ok, "offered_rate_hz": rate_hz,
            "solves_per_s": m / ((last - first) / 1e3), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_n": corr / m,
            "Mcorr_per_s": corr / ((last - first) / 1e3) / 1e6, "wall_s": wall,
            "budget_gb": budget_gb, "pool_problems": pool,
            "saturated_requests": len(seq), "saturated_in_flight": in_flight,
            "saturated_solves_per_s": len(seq) / sat_wall,
            "saturated_ok": sum(1 for r in sat if r["status"] == 0),
            "saturated_p50_ms": float(np.percentile(sat_lat, 50)),
            "saturated_p99_ms": float(np.percentile(sat_lat, 99)),
            "saturated_Mcorr_per_s": sat_corr / sat_wall / 1e6,
            "loop_solves_per_s": len(seq) / loop_wall,
            "saturated_vs_loop": loop_wall / sat_wall,
            "device_batches_solves_per_s": len(seq) / ceiling_wall,
            "loop_same_results": bool(same),
            "note": "host inputs (pageable numpy) on every path; the loop calls "
                    "sprot_estimate_rotations_k with HOST_PTRS once per request"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_sprot(args)


if __name__ == "__main__":
    main()
