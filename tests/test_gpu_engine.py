"""Fixpoint parity of the CUDA engine (through the C-ABI) with the CPU oracle:
identical sorted relations and identical per-iteration delta counts."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2311_02206_gb300 import workloads
from hisa_testutil import assert_same, assert_strictly_increasing_device, fingerprint_device, gpu_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


def modes():
    """host-driven, graph-captured, both with the log-structured full,
    graph-captured without the grouped bitmap join, and with hashed indexes,
    with Tmp joined and sorted instead of gathered, without pull mode, with a
    leveled full, and with the grouped bitmap join instead of the bit-matrix
    evaluation of REACH's shape"""
    from paper_2311_02206_gb300 import hisa
    return [0, hisa.FLAG_GRAPH, hisa.FLAG_LOG_FULL, hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL,
            hisa.FLAG_GRAPH | hisa.FLAG_NO_DENSE, hisa.FLAG_GRAPH | hisa.FLAG_NO_DENSE | hisa.FLAG_HASH_INDEX,
            hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL | hisa.FLAG_NO_CHAIN,
            hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL | hisa.FLAG_NO_PULL,
            hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL | hisa.FLAG_LEVELS,
            hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL | hisa.FLAG_NO_BITJOIN]


@pytest.mark.parametrize("ratio", [1 / 16, 4.0, 4096.0])
@pytest.mark.parametrize("graph", ["er1000", "rmat10", "path", "cycle", "star"] + [f"random{i}" for i in range(8)])
def test_reach_pull_switch_points(ratio, graph):
    """Groups pulled almost always (ratio 1/16), by the default rule, and
    never (4096): the same relation and delta counts as the oracle."""
    from paper_2311_02206_gb300 import hisa
    if graph == "er1000":
        s, d = workloads.config_reach_er()
    elif graph == "rmat10":
        s, d = workloads.rmat_graph(10, 1 << 13, 5)
    elif graph == "path":
        s, d = workloads.path_graph(200)
    elif graph == "cycle":
        s, d = workloads.cycle_graph(100)
    elif graph == "star":   # a hub with every edge in and out, plus a tail
        n = 300
        s = np.concatenate([np.arange(1, n), np.zeros(n - 1), np.arange(n, n + 50)]).astype(np.uint32)
        d = np.concatenate([np.zeros(n - 1), np.arange(1, n), np.arange(n + 1, n + 51)]).astype(np.uint32)
    else:
        rng = np.random.default_rng(100 + int(graph[6:]))
        n = int(rng.integers(2, 400))
        m = int(rng.integers(1, 6 * n))
        s = rng.integers(0, n, m).astype(np.uint32)
        d = rng.integers(0, n, m).astype(np.uint32)
    ref = oracle.reach(s, d)
    for flags in (hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL, hisa.FLAG_LOG_FULL):   # the grouped join's pull mode
        rels, counts, _ = gpu_eval(*oracle.REACH, {"Edge": (s, d)}, flags=flags | hisa.FLAG_NO_BITJOIN,
                                   pull_ratio=ratio)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("n", [3, 40, 700, 2000, 40000])
def test_reach_bitjoin_taken_and_exact(n):
    """A program of REACH's shape runs on bit matrices by default (its kernels
    are the ones launched) and on the grouped bitmap join with
    HISA_FLAG_NO_BITJOIN; both give the oracle's relation and delta counts.
    Domains from 2 to 16 bits: rows of one word, of fewer than one chunk, of
    one and of 32 chunks of 32 words."""
    from paper_2311_02206_gb300 import hisa
    rng = np.random.default_rng(n)
    m = 3 * n if n < 10000 else n + n // 2
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    if n >= 10000:   # keep the oracle quick: chains of 20 nodes over the whole domain
        s = np.arange(0, n - 1, dtype=np.uint32)
        s = s[(s % 20) != 19]
        d = s + 1
    ref = oracle.reach(s, d)
    for flags, bit in ((hisa.FLAG_PHASE_TIMES, True), (hisa.FLAG_PHASE_TIMES | hisa.FLAG_NO_BITJOIN, False)):
        with hisa.Context(flags=flags) as ctx:
            ctx.program(*oracle.REACH)
            ctx.load_tuples("Edge", s, d)
            ctx.run()
            names = {e["name"] for e in ctx.kernel_stats() if e["launches"] > 0}
            assert ("bit_join" in names or "bit_init" in names) == bit, names
            rels = {"Reach": ctx.read_relation("Reach")}
            counts = {"Reach": ctx.delta_counts("Reach")}
        assert_same(rels, counts, ref)


def test_bitjoin_two_base_rules_and_another_inner():
    """R(x, y) <- A(x, y); R(x, y) <- C(x, y); R(x, z) <- B(x, y), R(y, z):
    iteration 1 is the union of A and C, the recursion joins B."""
    from paper_2311_02206_gb300 import hisa
    rng = np.random.default_rng(11)
    n = 300
    edb = {k: (rng.integers(0, n, 400).astype(np.uint32), rng.integers(0, n, 400).astype(np.uint32))
           for k in ("A", "B", "C")}
    prog = ({"A": "edb", "B": "edb", "C": "edb", "R": "idb"},
            [(("R", ("x", "y")), [("A", ("x", "y"))], []),
             (("R", ("x", "y")), [("C", ("x", "y"))], []),
             (("R", ("x", "z")), [("R", ("y", "z")), ("B", ("x", "y"))], [])])
    ref = oracle.seminaive(*prog, edb)
    for flags in (hisa.FLAG_PHASE_TIMES, hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL | hisa.FLAG_NO_BITJOIN):
        rels, counts, _ = gpu_eval(*prog, edb, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("seed", range(40))
def test_reach_random_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 60))
    m = int(rng.integers(1, 4 * n))
    s = rng.integers(0, n, m).astype(np.uint32)          # repeats and self-loops included
    d = rng.integers(0, n, m).astype(np.uint32)
    ref = oracle.reach(s, d)
    for flags in modes():
        rels, counts, _ = gpu_eval(*oracle.REACH, {"Edge": (s, d)}, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("shape,n", [("path", 300), ("cycle", 64), ("dag", 120), ("path", 2)])
@pytest.mark.parametrize("log_full", [False, True])
def test_reach_closed_forms(shape, n, log_full):
    from paper_2311_02206_gb300 import hisa
    src, dst = {"path": workloads.path_graph, "cycle": workloads.cycle_graph,
                "dag": workloads.complete_dag}[shape](n)
    rels, counts, st = gpu_eval(*oracle.REACH, {"Edge": (src, dst)},
                                flags=hisa.FLAG_GRAPH | (hisa.FLAG_LOG_FULL if log_full else 0))
    size = len(rels["Reach"][0])
    if shape == "path":
        assert size == n * (n - 1) // 2 and counts["Reach"] == [n - k for k in range(1, n)]
    elif shape == "cycle":
        assert size == n * n and counts["Reach"] == [n] * n
    else:
        assert size == n * (n - 1) // 2 and counts["Reach"] == [n * (n - 1) // 2]


def test_reach_er_1000():
    """REACH on the ER graph n=1,000, m=3,000 (seed 0): the whole relation."""
    s, d = workloads.config_reach_er()
    ref = oracle.reach(s, d)
    for flags in modes():
        rels, counts, st = gpu_eval(*oracle.REACH, {"Edge": (s, d)}, flags=flags)
        assert_same(rels, counts, ref)
    assert ref.size("Reach") == 889_271


@pytest.mark.parametrize("prog", ["reach", "sg", "cspa"])
def test_read_relation_destinations(prog):
    """Each read path -- a column-swapped append-only full through the bit-matrix
    transpose (REACH), one in declared order through the level merge (SG), a
    single sorted full (the points-to program) -- gives the oracle's tuples in
    lexicographic order into page-locked host columns (staged or written over
    the host link), into pageable numpy arrays and into device tensors."""
    from paper_2311_02206_gb300 import hisa
    if prog == "reach":
        program, edb = oracle.REACH, {"Edge": workloads.config_reach_er()}
    elif prog == "sg":
        program, edb = oracle.SG, {"Edge": workloads.dag_graph(400, 900, 16, 3)}
    else:
        program, edb = oracle.CSPA, workloads.config_cspa(1000, 32)
    ref = oracle.reach(*edb["Edge"]) if prog == "reach" else oracle.seminaive(*program, edb)
    with hisa.Context() as ctx:
        ctx.program(*program)
        for k, (c0, c1) in edb.items():
            ctx.load_tuples(k, c0, c1)
        ctx.run()
        for name, (r0, r1) in ref.relations.items():
            n = ctx.relation_size(name)
            assert n == len(r0), name
            h0 = torch.empty(max(n, 1), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
            h1 = torch.empty(max(n, 1), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
            p0, p1 = ctx.read_relation(name, out=(h0, h1))
            a0, a1 = ctx.read_relation(name)
            d0, d1 = ctx.read_relation(name, device=True)
            for g0, g1 in ((p0, p1), (a0, a1), (d0.cpu().numpy().view(np.uint32), d1.cpu().numpy().view(np.uint32))):
                assert np.array_equal(g0, r0) and np.array_equal(g1, r1), name


def test_reach_wide_codes():
    """Node ids spread over the full uint32 range (64-bit codes, b = 32)."""
    rng = np.random.default_rng(11)
    s = rng.integers(0, 50, 120).astype(np.uint64)
    d = rng.integers(0, 50, 120).astype(np.uint64)
    relabel = (np.arange(50, dtype=np.uint64) * np.uint64(0x9E3779B1) + np.uint64(0xFFFF0000)) % np.uint64(1 << 32)
    relabel[0] = 0xFFFFFFFF
    s, d = relabel[s].astype(np.uint32), relabel[d].astype(np.uint32)
    ref = oracle.reach(s, d)
    rels, counts, _ = gpu_eval(*oracle.REACH, {"Edge": (s, d)})
    assert_same(rels, counts, ref)


def test_reach_empty_and_single():
    e = np.zeros(0, np.uint32)
    rels, counts, st = gpu_eval(*oracle.REACH, {"Edge": (e, e)})
    assert len(rels["Reach"][0]) == 0 and counts["Reach"] == []
    one = np.array([3], np.uint32)
    rels, counts, st = gpu_eval(*oracle.REACH, {"Edge": (one, one)})
    assert rels["Reach"][0].tolist() == [3] and counts["Reach"] == [1]


def test_reach_deterministic_and_reusable():
    from paper_2311_02206_gb300 import hisa
    s, d = workloads.er_graph(400, 1200, 7)
    with hisa.Context() as ctx:
        ctx.program(*oracle.REACH)
        ctx.load_tuples("Edge", s, d)
        ctx.run()
        a = ctx.read_relation("Reach"), ctx.delta_counts("Reach")
        ctx.run()
        b = ctx.read_relation("Reach"), ctx.delta_counts("Reach")
    assert np.array_equal(a[0][0], b[0][0]) and np.array_equal(a[0][1], b[0][1]) and a[1] == b[1]


def test_load_from_device_tensors():
    from paper_2311_02206_gb300 import hisa
    s, d = workloads.er_graph(300, 900, 3)
    ref = oracle.reach(s, d)
    with hisa.Context() as ctx:
        ctx.program(*oracle.REACH)
        half = len(s) // 2
        ctx.load_tuples("Edge", torch.from_numpy(s[:half].view(np.int32)).cuda(),
                        torch.from_numpy(d[:half].view(np.int32)).cuda())
        ctx.load_tuples("Edge", s[half:], d[half:])
        ctx.run()
        c0, c1 = ctx.read_relation("Reach", device=True)
        assert np.array_equal(c0.cpu().numpy().view(np.uint32), ref.relations["Reach"][0])
        assert np.array_equal(c1.cpu().numpy().view(np.uint32), ref.relations["Reach"][1])


def test_not_converged_and_budget_errors():
    from paper_2311_02206_gb300 import hisa
    s, d = workloads.path_graph(50)
    with hisa.Context(max_iters=10) as ctx:
        ctx.program(*oracle.REACH)
        ctx.load_tuples("Edge", s, d)
        with pytest.raises(hisa.HisaError) as e:
            ctx.run()
        assert e.value.status == -4
    with hisa.Context(hbm_budget_bytes=1 << 20) as ctx:
        ctx.program(*oracle.REACH)
        with pytest.raises(hisa.HisaError) as e:
            ctx.load_tuples("Edge", *workloads.er_graph(2000, 8000, 1))
            ctx.run()
        assert e.value.status == -3


@pytest.mark.parametrize("depth", [3, 6])
def test_sg_binary_tree(depth):
    rels, counts, _ = gpu_eval(*oracle.SG, {"Edge": workloads.binary_tree(depth)})
    ref = oracle.seminaive(*oracle.SG, {"Edge": workloads.binary_tree(depth)})
    assert_same(rels, counts, ref)


@pytest.mark.parametrize("seed", range(6))
def test_sg_random_dag(seed):
    s, d = workloads.dag_graph(300, 700, 16, seed)
    ref = oracle.seminaive(*oracle.SG, {"Edge": (s, d)})
    for flags in modes():
        rels, counts, _ = gpu_eval(*oracle.SG, {"Edge": (s, d)}, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("log_full,no_dense,no_pull,levels,no_bitjoin",
                         [(False, True, False, False, False), (True, True, False, False, False),
                          (True, False, False, False, False), (True, False, True, False, False),
                          (True, False, False, True, False), (True, False, False, False, True)])
def test_reach_rmat_full_size_golden_and_sampled(log_full, no_dense, no_pull, levels, no_bitjoin):
    """REACH on R-MAT scale 16 / 2**19 edges, in the launch configuration the
    benchmark times: total size, delta counts and fingerprint against the
    oracle's stored values, and 16 sampled target columns element by element."""
    path = os.path.join(GOLDEN, "reach_rmat_s16.json")
    if not os.path.exists(path):
        pytest.skip("golden values not generated")
    g = json.load(open(path))
    from paper_2311_02206_gb300 import hisa
    s, d = workloads.config_reach_rmat()
    flags = hisa.FLAG_GRAPH | (hisa.FLAG_LOG_FULL if log_full else 0) | (hisa.FLAG_NO_DENSE if no_dense else 0) | \
        (hisa.FLAG_NO_PULL if no_pull else 0) | (hisa.FLAG_LEVELS if levels else 0) | \
        (hisa.FLAG_NO_BITJOIN if no_bitjoin else 0)
    with hisa.Context(flags=flags) as ctx:
        ctx.program(*oracle.REACH)
        ctx.load_tuples("Edge", s, d)
        ctx.run()
        assert ctx.delta_counts("Reach") == g["delta_counts"]
        assert ctx.relation_size("Reach") == g["reach_size"]
        c0, c1 = ctx.read_relation("Reach", device=True)
        assert fingerprint_device(c0, c1) == int(g["fingerprint"])
        assert_strictly_increasing_device(c0, c1)
        targets = np.random.default_rng(2024).choice(1 << 16, 16, replace=False).astype(np.uint32)
        ref = oracle.reach_targets(s, d, targets)
        keep = torch.isin(c1, torch.from_numpy(targets.view(np.int32)).cuda())
        g0 = c0[keep].cpu().numpy().view(np.uint32)
        g1 = c1[keep].cpu().numpy().view(np.uint32)
        assert np.array_equal(g0, ref.relations["Reach"][0]) and np.array_equal(g1, ref.relations["Reach"][1])


_SG_SUB = {}


def _sg_induced(literal, nodes):
    """The oracle's SG on the subgraph of the 20,000-node DAG induced by the
    nodes [0, nodes).  Edges point to larger ids, so every derivation of SG(x,
    y) with x, y < nodes (rule 1 through a parent p < x, rule 2 through a, b <
    x, y) uses nodes below `nodes` only: this is exactly SG restricted to
    [0, nodes)^2."""
    key = (literal, nodes)
    if key not in _SG_SUB:
        s, d = workloads.config_sg_dag()
        keep = (s < nodes) & (d < nodes)
        _SG_SUB[key] = oracle.seminaive(*(oracle.SG_LITERAL if literal else oracle.SG),
                                        {"Edge": (s[keep], d[keep])}).relations["SG"]
    return _SG_SUB[key]


@pytest.mark.parametrize("literal,log_full,no_chain,levels",
                         [(False, False, False, False), (True, False, False, False), (False, True, False, False),
                          (False, True, True, False), (False, True, False, True)])
def test_sg_dag_full_size_golden(literal, log_full, no_chain, levels):
    """SG on the 20,000-node DAG (x != y on both rules, or on rule 1 only as
    the workload description prints it): size, every delta count and the
    fingerprint of the whole relation against the oracle's stored values; the
    whole relation in strictly increasing order; and, element by element and
    position by position, its restriction to nodes [0, 3000) against the
    oracle's SG of the induced subgraph (3.1 million tuples)."""
    path = os.path.join(GOLDEN, "sg_literal_dag_20k.json" if literal else "sg_dag_20k.json")
    if not os.path.exists(path):
        pytest.skip("golden values not generated")
    g = json.load(open(path))
    from paper_2311_02206_gb300 import hisa
    s, d = workloads.config_sg_dag()
    flags = hisa.FLAG_GRAPH | (hisa.FLAG_LOG_FULL if log_full else 0) | (hisa.FLAG_NO_CHAIN if no_chain else 0) | \
        (hisa.FLAG_LEVELS if levels else 0)
    with hisa.Context(flags=flags) as ctx:
        ctx.program(*(oracle.SG_LITERAL if literal else oracle.SG))
        ctx.load_tuples("Edge", s, d)
        ctx.run()
        assert ctx.delta_counts("SG") == g["delta_counts"]
        assert ctx.relation_size("SG") == g["sg_size"]
        c0, c1 = ctx.read_relation("SG", device=True)
        assert fingerprint_device(c0, c1) == int(g["fingerprint"])
        assert_strictly_increasing_device(c0, c1)
        nodes = 3000
        keep = (c0 >= 0) & (c0 < nodes) & (c1 >= 0) & (c1 < nodes)
        g0 = c0[keep].cpu().numpy().view(np.uint32)
        g1 = c1[keep].cpu().numpy().view(np.uint32)
    w0, w1 = _sg_induced(literal, nodes)
    assert len(w0) > 3_000_000
    assert np.array_equal(g0, w0) and np.array_equal(g1, w1)


def _cspa_arrays(div, window):
    path = os.path.join(GOLDEN, "cspa_d%d_w%d.npz" % (div, window))
    if not os.path.exists(path):
        return None
    z = np.load(path)
    return {k: ((z[k] >> np.uint64(32)).astype(np.uint32), (z[k] & np.uint64(0xFFFFFFFF)).astype(np.uint32))
            for k in z.files}


@pytest.mark.parametrize("div,window,no_chain", [(500, 32, False), (250, 128, False), (500, 32, True)])
def test_cspa_golden(div, window, no_chain):
    """The points-to program on the skewed inputs divided by `div`: sizes,
    delta counts and fingerprints of the three IDB relations against the
    oracle's stored values, and every tuple of each relation, in order,
    against the oracle's stored sorted relations (1/250 derives ~4.6e9 raw
    tuples on the GPU)."""
    path = os.path.join(GOLDEN, "cspa_d%d_w%d.json" % (div, window))
    if not os.path.exists(path):
        pytest.skip("golden values not generated")
    g = json.load(open(path))
    arrays = _cspa_arrays(div, window)
    from paper_2311_02206_gb300 import hisa
    edb = workloads.config_cspa(div, window)
    flags = hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL | (hisa.FLAG_NO_CHAIN if no_chain else 0)
    with hisa.Context(flags=flags) as ctx:
        ctx.program(*oracle.CSPA)
        for name, (c0, c1) in edb.items():
            ctx.load_tuples(name, c0, c1)
        st = ctx.run()
        assert st.iterations == g["iterations"]
        for name in ("ValueFlow", "MemoryAlias", "ValueAlias"):
            assert ctx.relation_size(name) == g[name]["size"], name
            assert ctx.delta_counts(name) == g[name]["delta_counts"], name
            c0, c1 = ctx.read_relation(name, device=True)
            assert fingerprint_device(c0, c1) == int(g[name]["fingerprint"]), name
            assert_strictly_increasing_device(c0, c1)
            if arrays is not None:
                w0, w1 = arrays[name]
                assert np.array_equal(c0.cpu().numpy().view(np.uint32), w0), name
                assert np.array_equal(c1.cpu().numpy().view(np.uint32), w1), name
    assert arrays is not None, "stored sorted relations missing (tests/golden/make_golden.py cspa)"


@pytest.mark.parametrize("knobs", [dict(radix_items=16), dict(radix_items=8), dict(dense_unit=64),
                                   dict(dense_unit=1024, pull_ratio=2.0), dict(load_factor=0.5)])
def test_tuning_knobs_keep_results(knobs):
    """Every value the autotuner may pick (radix tile, join work split, pull
    switch point, load factor of the hashed index) gives the oracle's
    relations and delta counts, on the sort path, the grouped join and the
    hashed indexes."""
    from paper_2311_02206_gb300 import hisa
    cases = [(oracle.REACH, {"Edge": workloads.config_reach_er()}),
             (oracle.SG, {"Edge": workloads.dag_graph(300, 700, 16, 4)}),
             (oracle.CSPA, workloads.config_cspa(1000, 32))]
    for prog, edb in cases:
        ref = oracle.seminaive(*prog, edb)
        for flags in (hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL, hisa.FLAG_GRAPH | hisa.FLAG_NO_DENSE,
                      hisa.FLAG_GRAPH | hisa.FLAG_HASH_INDEX | hisa.FLAG_LOG_FULL):
            rels, counts, _ = gpu_eval(*prog, edb, flags=flags, **knobs)
            assert_same(rels, counts, ref)

