"""The bench's reference arm without a GPU (not gpu): `bench.py --impl reference` times the FP64
oracle on the host's cores and prints one JSON line on the same metric, unit and workload as
the library's arm, with its CPU sample described, and an e2e entry that moves no bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    sys.path.insert(0, ROOT)
    import bench

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    r = json.loads(lines[0])
    assert r["impl"] == "reference"
    assert r["metric"] == bench.METRIC and r["unit"] == bench.UNIT == "Mcorr/s"
    assert r["config"]["workload"] == bench.WORKLOAD
    assert (r["config"]["n"], r["config"]["grid"], r["config"]["angle_bins"]) == (1_000_000, 512, 720)
    assert r["higher_is_better"] is True and r["n_gpus"] == 1
    assert (r["steps"], r["warmup"]) == (1, 3)
    assert r["value"] > 0 and r["ms_per_step"] > 0
    assert r["dtype"] == "f64" and r["vs_baseline"] is None
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": "Mcorr/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_two_ranks_prints_once():
    """Launched for N = 2 with torchrun (one process per rank): rank 0 alone runs the oracle and
    prints the line, with n_gpus = 2; the other rank exits 0 without work."""
    import socket

    with socket.socket() as sk:  # a free port for the rendezvous
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["n_gpus"] == 2 and r["value"] > 0


def test_vote_traffic_record_is_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    """The roofline's `traffic` comes from the committed ncu record of the axis-vote kernel only
    while the kernel's source is the one the counters were taken on (its sha256); a changed
    source gives no record, so the line reports traffic null."""
    import hashlib
    import shutil

    sys.path.insert(0, ROOT)
    import bench

    rec = json.load(open(os.path.join(ROOT, "profiles", "axis_vote_traffic.json")))
    assert rec["workload"] == bench.WORKLOAD
    for key in ("dram_bytes_per_launch", "warp_instructions_per_launch", "grid_ctas", "command"):
        assert key in rec
    # a copy of the tree with the record and the kernel source
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2502_06337_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "axis_vote_traffic.json"), tmp_path / "profiles")
    src = tmp_path / "paper_2502_06337_gb300" / "csrc" / "vote_runs.cu"
    shutil.copy(os.path.join(ROOT, "paper_2502_06337_gb300", "csrc", "vote_runs.cu"), src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    same = hashlib.sha256(src.read_bytes()).hexdigest() == rec["kernel_source_sha256"]
    assert bench.vote_profile() == (rec if same else {})
    src.write_bytes(src.read_bytes() + b"\n// changed\n")
    assert bench.vote_profile() == {}
