"""The hash-partitioned REACH (paper_2311_02206_gb300.partitioned) on CPU:
its iteration and exchange logic with the per-partition steps written from
the oracle's definitions, on world_size 2 and 3 gloo ranks (the all-to-all and
all-reduce of torch.distributed) and on several partitions in one process.
The union of the ranks' parts must be the oracle's Reach, every tuple must sit
on the owner of its first column, and the delta counts summed over the ranks
must be the oracle's."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2311_02206_gb300 import partitioned, workloads
from partition_testutil import OracleOps, decode, owner

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _graphs():
    rng = np.random.default_rng(41)
    out = {"path": workloads.path_graph(40), "cycle": workloads.cycle_graph(23), "dag": workloads.complete_dag(15),
           "er": workloads.er_graph(120, 300, 3), "single": (np.array([3], np.uint32), np.array([3], np.uint32))}
    for i in range(3):
        n = int(rng.integers(2, 80))
        m = int(rng.integers(1, 4 * n))
        out[f"random{i}"] = (rng.integers(0, n, m).astype(np.uint32), rng.integers(0, n, m).astype(np.uint32))
    return out


def _split(s, d, parts):
    """Edge list cut into `parts` contiguous shares (any split works)."""
    cuts = np.linspace(0, len(s), parts + 1).astype(int)
    return [(torch.from_numpy(s[cuts[p]:cuts[p + 1]].view(np.int32).copy()),
             torch.from_numpy(d[cuts[p]:cuts[p + 1]].view(np.int32).copy())) for p in range(parts)]


def _check(parts_full, b, counts, s, d, nparts):
    ref = oracle.reach(s, d)
    w0, w1 = ref.relations["Reach"]
    got = np.sort(np.concatenate([f.numpy().astype(np.uint64) for f in parts_full]))
    g0, g1 = decode(got, b)
    assert np.array_equal(g0, w0) and np.array_equal(g1, w1)
    assert counts == ref.delta_counts["Reach"]
    for p, f in enumerate(parts_full):
        c0, _ = decode(f.numpy().astype(np.uint64), b)
        assert np.all(owner(c0, nparts) == p), "a tuple sits on a rank that does not own its first column"
        assert np.all(np.diff(f.numpy()) > 0), "a part is not sorted and duplicate-free"


@pytest.mark.parametrize("nparts", [1, 2, 5])
def test_partitioned_reach_local_partitions(nparts):
    for name, (s, d) in _graphs().items():
        full, b, counts = partitioned.reach_partitioned(_split(s, d, nparts), OracleOps(),
                                                        partitioned.LocalExchange(nparts))
        _check(full, b, counts, s, d, nparts)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2311_02206_gb300 import partitioned as pt
    from partition_testutil import OracleOps as Ops
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        out = {}
        for name, (s, d) in _graphs().items():
            share = _split(s, d, world)[rank]
            full, b, counts = pt.reach_partitioned([share], Ops(), pt.TorchExchange())
            out[name] = (full[0].numpy().copy(), b, counts)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_reach_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for name, (s, d) in _graphs().items():
        parts = [torch.from_numpy(results[r][name][0]) for r in range(world)]
        b = results[0][name][1]
        counts = results[0][name][2]
        assert all(results[r][name][1:] == (b, counts) for r in range(world))
        _check(parts, b, counts, s, d, world)
