"""bench.py's multi-rank timing on CPU: two gloo ranks (the layout torchrun
gives one rank per GPU) reduce their timed-region lengths to the maximum and
report the whole-job rate.  The path itself needs no exchange (replicas), so
this is the only collective bench.py performs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.env_rank() == (rank, world, rank)
        ms, rate = bench.whole_job_rate(100.0 * (rank + 1), steps=10, world=world, device="cpu")
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, rate in out:
        assert ms == 200.0                      # the slower rank's 200 ms
        assert rate == pytest.approx(2 * 10 / 0.2)  # 2 ranks x 10 steps in 0.2 s


def test_single_rank_needs_no_process_group():
    import bench
    ms, rate = bench.whole_job_rate(250.0, steps=5, world=1)
    assert ms == 250.0 and rate == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle arm is timed and printed by rank 0 alone;
    the other ranks return at once without work or output."""
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(argparse.Namespace(steps=1, warmup=3, gpus=2))
    assert capsys.readouterr().out == ""
