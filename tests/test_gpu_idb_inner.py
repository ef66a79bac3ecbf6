"""Programs whose IDB relations are range-probed inner relations: the index over
full (column 0) and the reverse-order mirror of full (column 1) are rebuilt
every iteration.  Parity with the oracle: identical sorted relations and
identical per-iteration delta counts, host-driven and graph-captured."""
import numpy as np
import pytest

import oracle
from paper_2311_02206_gb300 import workloads
from hisa_testutil import assert_same, gpu_eval
from programs import INVERTED, MUTUAL, TC_NONLINEAR

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


def modes():
    """host-driven and graph-captured; graph-captured with hashed indexes, and
    with Tmp joined and sorted instead of gathered"""
    from paper_2311_02206_gb300 import hisa
    return [0, hisa.FLAG_GRAPH, hisa.FLAG_GRAPH | hisa.FLAG_HASH_INDEX, hisa.FLAG_GRAPH | hisa.FLAG_NO_CHAIN]


def random_graph(seed, nmax=60, dmax=4):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, nmax))
    m = int(rng.integers(1, dmax * n))
    return rng.integers(0, n, m).astype(np.uint32), rng.integers(0, n, m).astype(np.uint32)


@pytest.mark.parametrize("seed", range(24))
def test_tc_nonlinear_random(seed):
    edb = {"E": random_graph(seed)}
    ref = oracle.seminaive(*TC_NONLINEAR, edb)
    for flags in modes():
        rels, counts, _ = gpu_eval(*TC_NONLINEAR, edb, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("shape,n", [("path", 700), ("cycle", 97), ("path", 2)])
def test_tc_nonlinear_closed_forms(shape, n):
    """Relations far above the initial capacities: full, its mirror and both
    indexes grow several times during the run."""
    g = workloads.path_graph(n) if shape == "path" else workloads.cycle_graph(n)
    ref = oracle.seminaive(*TC_NONLINEAR, {"E": g})
    for flags in modes():
        rels, counts, st = gpu_eval(*TC_NONLINEAR, {"E": g}, flags=flags)
        assert_same(rels, counts, ref)
    assert len(rels["T"][0]) == (n * (n - 1) // 2 if shape == "path" else n * n)


def test_tc_nonlinear_wide_codes():
    """Values up to 2**20: 64-bit codes."""
    s, d = random_graph(7, nmax=300, dmax=2)
    s = (s.astype(np.uint64) * 3511 % (1 << 20)).astype(np.uint32)
    d = (d.astype(np.uint64) * 3511 % (1 << 20)).astype(np.uint32)
    ref = oracle.seminaive(*TC_NONLINEAR, {"E": (s, d)})
    for flags in modes():
        rels, counts, _ = gpu_eval(*TC_NONLINEAR, {"E": (s, d)}, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("seed", range(24))
def test_mutual_random(seed):
    edb = {"A": random_graph(2 * seed, 30, 3), "B": random_graph(2 * seed + 1, 30, 3)}
    ref = oracle.seminaive(*MUTUAL, edb)
    for flags in modes():
        rels, counts, _ = gpu_eval(*MUTUAL, edb, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("seed", range(16))
def test_inverted_filter_random(seed):
    """x != y in a rule run as an inverted grouped bitmap join by default, and
    as a join + sort with HISA_FLAG_NO_CHAIN (one of the modes)."""
    edb = {"E": random_graph(3 * seed + 1, 50, 3)}
    ref = oracle.seminaive(*INVERTED, edb)
    for flags in modes():
        rels, counts, _ = gpu_eval(*INVERTED, edb, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("seed", range(12))
def test_cspa_tiny(seed):
    edb = workloads.cspa_inputs(25 + seed, 12, 14, window=4, seed=seed)
    ref = oracle.seminaive(*oracle.CSPA, edb)
    for flags in modes():
        rels, counts, _ = gpu_eval(*oracle.CSPA, edb, flags=flags)
        assert_same(rels, counts, ref)


@pytest.mark.parametrize("args", [(120, 60, 90, 16, 3), (250, 120, 180, 16, 4), (400, 200, 300, 32, 5)])
def test_cspa_small(args):
    """Skewed (Zipf 1.1) ids, windows of 16-32 ids: thousands of tuples in the
    three IDB relations over 8-11 iterations."""
    na, nd, ids, win, seed = args
    edb = workloads.cspa_inputs(na, nd, ids, window=win, seed=seed)
    ref = oracle.seminaive(*oracle.CSPA, edb)
    for flags in modes():
        rels, counts, _ = gpu_eval(*oracle.CSPA, edb, flags=flags)
        assert_same(rels, counts, ref)


def test_tc_nonlinear_batched_and_served():
    """Static batch and a serving session (retirement compacts full and its
    mirror) with the non-linear closure: each instance equals its run alone."""
    from paper_2311_02206_gb300 import hisa
    graphs = [random_graph(100 + i, 40, 3) for i in range(20)]
    refs = [oracle.seminaive(*TC_NONLINEAR, {"E": g}) for g in graphs]

    def check(ref, c0, c1, counts):
        w0, w1 = ref.relations["T"]
        assert np.array_equal(c0, w0) and np.array_equal(c1, w1)
        assert counts == ref.delta_counts["T"]

    with hisa.Context() as ctx:
        ctx.program(*TC_NONLINEAR)
        for i, g in enumerate(graphs):
            ctx.load_instance("E", i, *g)
        ctx.run()
        for i, ref in enumerate(refs):
            c0, c1 = ctx.read_instance("T", i)
            check(ref, c0, c1, ctx.instance_delta_counts("T", i))
    with hisa.Context() as ctx:
        ctx.program(*TC_NONLINEAR)
        ctx.serve_open(6, 63)
        tickets = {ctx.serve_submit("E", *g): i for i, g in enumerate(graphs[:12])}
        steps = 0
        while True:
            st = ctx.serve_step(1)
            steps += 1
            if steps == 3:
                for i in range(12, 20):
                    tickets[ctx.serve_submit("E", *graphs[i])] = i
            if steps > 3 and st["active"] == 0 and st["pending"] == 0:
                break
            assert steps < 1000
        for t, i in tickets.items():
            c0, c1, counts = ctx.serve_result(t, "T")
            check(refs[i], c0, c1, counts)
