"""The multi-GPU building blocks through the C-ABI (hisa_encode_codes,
hisa_decode_codes, hisa_column_max, hisa_partition_codes) against numpy and
the oracle's owner function, and the hash-partitioned REACH with its CUDA
steps on one GPU: several partitions held by one process (the all-to-all is
slicing), and one rank of a one-process NCCL group (the real all_to_all_single
and all_reduce), each against the oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2311_02206_gb300 import workloads
from partition_testutil import decode, owner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.mark.parametrize("n,b,wide", [(0, 5, False), (1, 1, False), (100_003, 16, False), (250_000, 20, True),
                                      (77, 32, True)])
def test_encode_decode_max(n, b, wide):
    from paper_2311_02206_gb300 import hisa
    rng = np.random.default_rng(n + b)
    c0 = rng.integers(0, 1 << b, n, dtype=np.uint64).astype(np.uint32)
    c1 = rng.integers(0, 1 << b, n, dtype=np.uint64).astype(np.uint32)
    codes = hisa.encode_codes(_dev(c0), _dev(c1), b, wide)
    want = (c0.astype(np.uint64) << np.uint64(b)) | c1.astype(np.uint64)
    got = codes.cpu().numpy().view(np.uint64 if wide else np.uint32).astype(np.uint64)
    assert np.array_equal(got, want)
    d0, d1 = hisa.decode_codes(codes, b)
    assert np.array_equal(d0.cpu().numpy().view(np.uint32), c0) and np.array_equal(d1.cpu().numpy().view(np.uint32), c1)
    mx = hisa.column_max(_dev(c0), _dev(c1))
    assert mx == (int(max(c0.max(), c1.max())) if n else 0)


@pytest.mark.parametrize("n,b,key_col,nparts", [(0, 8, 0, 4), (5, 8, 1, 1), (1_000_003, 16, 0, 8),
                                                (300_001, 16, 1, 3), (200_000, 24, 0, 1024), (99_999, 30, 1, 7)])
def test_partition_codes_groups_by_owner(n, b, key_col, nparts):
    from paper_2311_02206_gb300 import hisa
    wide = 2 * b > 32
    rng = np.random.default_rng(n + nparts)
    c0 = rng.integers(0, 1 << b, n, dtype=np.uint64).astype(np.uint32)
    c1 = rng.integers(0, 1 << b, n, dtype=np.uint64).astype(np.uint32)
    c1[: n // 3] = 7   # many equal keys
    codes = hisa.encode_codes(_dev(c0), _dev(c1), b, wide)
    out, counts = hisa.partition_codes(codes, b, key_col, nparts)
    own = owner(c0 if key_col == 0 else c1, nparts)
    assert counts == np.bincount(own, minlength=nparts).tolist()
    got = out.cpu().numpy().view(np.uint64 if wide else np.uint32).astype(np.uint64)
    src = codes.cpu().numpy().view(np.uint64 if wide else np.uint32).astype(np.uint64)
    lo = 0
    for p in range(nparts):
        part = got[lo:lo + counts[p]]
        assert np.array_equal(np.sort(part), np.sort(src[own == p])), p
        lo += counts[p]


def _graphs():
    rng = np.random.default_rng(7)
    out = {"er1000": workloads.config_reach_er(), "rmat10": workloads.rmat_graph(10, 1 << 13, 3),
           "cycle": workloads.cycle_graph(50), "path": workloads.path_graph(120),
           "wide": (np.array([0xFFFFFFFF, 5, 9], np.uint32), np.array([5, 9, 0xFFFFFFFF], np.uint32))}
    for i in range(4):
        n = int(rng.integers(2, 500))
        m = int(rng.integers(1, 5 * n))
        out[f"random{i}"] = (rng.integers(0, n, m).astype(np.uint32), rng.integers(0, n, m).astype(np.uint32))
    return out


_REF = {}


def _check(full, b, counts, s, d, nparts):
    key = (s.tobytes(), d.tobytes())
    if key not in _REF:
        _REF[key] = oracle.reach(s, d)
    ref = _REF[key]
    w0, w1 = ref.relations["Reach"]
    from paper_2311_02206_gb300 import hisa
    parts = []
    for p, f in enumerate(full):
        c0, c1 = (x.cpu().numpy().view(np.uint32) for x in hisa.decode_codes(f, b))
        assert np.all(owner(c0, nparts) == p)
        parts.append((c0.astype(np.uint64) << np.uint64(32)) | c1.astype(np.uint64))
    allc = np.concatenate(parts) if parts else np.zeros(0, np.uint64)
    order = np.argsort(allc, kind="stable")
    g0, g1 = decode(allc[order], 32)
    assert np.array_equal(g0, w0) and np.array_equal(g1, w1)
    assert counts == ref.delta_counts["Reach"]


@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
def test_partitioned_reach_on_one_gpu(nparts):
    from paper_2311_02206_gb300 import partitioned
    for name, (s, d) in _graphs().items():
        cuts = np.linspace(0, len(s), nparts + 1).astype(int)
        edges = [(_dev(s[cuts[p]:cuts[p + 1]]), _dev(d[cuts[p]:cuts[p + 1]])) for p in range(nparts)]
        full, b, counts = partitioned.reach_partitioned(edges, partitioned.CudaPartOps(),
                                                        partitioned.LocalExchange(nparts))
        _check(full, b, counts, s, d, nparts)


_NCCL_CHILD = r"""
import os, sys
import numpy as np, torch, torch.distributed as dist
sys.path.insert(0, ROOT); sys.path.insert(0, os.path.join(ROOT, "tests"))
from paper_2311_02206_gb300 import partitioned, workloads
torch.cuda.set_device(0)
dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % PORT, rank=0, world_size=1)
s, d = workloads.config_reach_er()
edges = [(torch.from_numpy(s.view(np.int32)).cuda(), torch.from_numpy(d.view(np.int32)).cuda())]
full, b, counts = partitioned.reach_partitioned(edges, partitioned.CudaPartOps(), partitioned.TorchExchange())
np.save(OUT, full[0].cpu().numpy())
print("B", b, "COUNTS", ",".join(map(str, counts)))
dist.destroy_process_group()
"""


def test_partitioned_reach_nccl_one_rank(tmp_path):
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "full.npy")
    code = _NCCL_CHILD.replace("ROOT", repr(ROOT)).replace("PORT", str(port)).replace("OUT", repr(out))
    env = dict(os.environ, NCCL_NVLS_ENABLE="0", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("B ")][-1].split()
    b, counts = int(line[1]), [int(x) for x in line[3].split(",")]
    s, d = workloads.config_reach_er()
    ref = oracle.reach(s, d)
    codes = np.load(out).view(np.uint32).astype(np.uint64)
    g0, g1 = decode(codes, b)
    w0, w1 = ref.relations["Reach"]
    assert np.array_equal(g0, w0) and np.array_equal(g1, w1)
    assert counts == ref.delta_counts["Reach"]
