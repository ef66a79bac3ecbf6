"""The N > 1 bench path on CPU: world_size-2 gloo ranks (no GPU).  bench.py
runs one independent replica per GPU (the path has no exchange step), so
the multi-rank logic is the barrier around the timed steps, the maximum of
the ranks' times and the sum of the ranks' tuples, and the reference arm
running on rank 0 alone."""
import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench._barrier(world)
        # a replica's time and tuples: rank r took 10 (r + 1) ms for 1000 (r + 1) tuples
        slowest = bench._max_over_ranks(0.010 * (rank + 1), world)
        tuples = bench._sum_over_ranks(1000.0 * (rank + 1), world)
        bench._barrier(world)
        out.put((rank, slowest, tuples))
    finally:
        dist.destroy_process_group()


def test_replica_reductions_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # whole-job value = all ranks' tuples / the slowest rank's time
    for rank, slowest, tuples in got:
        assert slowest == pytest.approx(0.020) and tuples == pytest.approx(3000.0)
        assert tuples / slowest == pytest.approx(150000.0)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    a = argparse.Namespace(workload="rmat16", steps=1, warmup=3, gpus=2)
    assert bench.run_reference(a) is None
    assert capsys.readouterr().out == ""
