"""The multi-process path of bench.py on CPU: two gloo ranks, as torchrun starts them.

bench.py runs one independent replica per GPU (the path has no data-path exchange); the job
time is the maximum over ranks and the throughput counts every rank's work. These tests run
its rank helpers with world_size 2 on the gloo backend."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    try:
        bench.barrier(w)
        t_job = bench.max_over_ranks(1.5 + r, w)  # rank 1 is the slow one
        bench.barrier(w)
        out.put((r, w, local, t_job))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_barrier():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 0, 2.5), (1, 2, 1, 2.5)]


def test_single_process_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench

    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.25, 1) == 3.25
    bench.barrier(1)  # no process group: a no-op


@pytest.mark.parametrize("world", [2, 4])
def test_reference_arm_runs_on_rank_zero_only(world, monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints; the other ranks exit at once."""
    import bench

    monkeypatch.setenv("WORLD_SIZE", str(world))
    monkeypatch.setenv("RANK", str(world - 1))
    monkeypatch.setenv("LOCAL_RANK", str(world - 1))
    args = type("A", (), dict(steps=1, warmup=0))()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
