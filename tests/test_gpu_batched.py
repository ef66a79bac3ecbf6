"""Batched and served evaluation of independent REACH instances: every
instance's tuples and delta counts must equal those of the oracle run on that
instance alone, whether it ran in a static batch or was admitted into (and
retired from) a running serving session."""
import numpy as np
import pytest

import oracle
from paper_2311_02206_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


def instances(count, seed, nmax=60):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(2, nmax))
        m = int(rng.integers(0, 3 * n))
        s = rng.integers(0, n, m).astype(np.uint32)
        d = rng.integers(0, n, m).astype(np.uint32)
        out.append((s, d))
    return out


def check(ref, c0, c1, counts):
    w0, w1 = ref.relations["Reach"]
    assert np.array_equal(c0, w0) and np.array_equal(c1, w1)
    assert counts == ref.delta_counts["Reach"]


def _full_modes():
    from paper_2311_02206_gb300 import hisa
    # 0: full as a bit matrix with a block of rows per instance; LEVELS: a
    # sorted full cut by instance
    return [0, hisa.FLAG_LEVELS]


@pytest.mark.parametrize("mode", [0, 1], ids=["matrix", "sorted"])
def test_static_batch_matches_each_instance_alone(mode):
    """Each instance alone, and the whole relation: relation_size is the sum of
    the instances' sizes and read_relation their tuples in instance order."""
    from paper_2311_02206_gb300 import hisa
    inst = instances(48, 1)
    with hisa.Context(flags=_full_modes()[mode]) as ctx:
        ctx.program(*oracle.REACH)
        for i, (s, d) in enumerate(inst):
            ctx.load_instance("Edge", i, s, d)
        ctx.run()
        all0, all1 = [], []
        for i, (s, d) in enumerate(inst):
            c0, c1 = ctx.read_instance("Reach", i)
            check(oracle.reach(s, d), c0, c1, ctx.instance_delta_counts("Reach", i))
            assert ctx.instance_size("Reach", i) == len(c0)
            all0.append(c0)
            all1.append(c1)
        assert ctx.relation_size("Reach") == sum(len(x) for x in all0)
        r0, r1 = ctx.read_relation("Reach")
        assert np.array_equal(r0, np.concatenate(all0)) and np.array_equal(r1, np.concatenate(all1))


@pytest.mark.parametrize("mode", [0, 1], ids=["matrix", "sorted"])
def test_serving_continuous_admission_and_slot_reuse(mode):
    """8 slots, 40 requests submitted in three waves while the session runs:
    requests wait for free slots, are admitted at iteration boundaries next to
    running ones, and slots of finished requests are reused (a reused slot's
    block of matrix rows starts empty)."""
    from paper_2311_02206_gb300 import hisa
    inst = instances(40, 2)
    with hisa.Context(flags=_full_modes()[mode]) as ctx:
        ctx.program(*oracle.REACH)
        ctx.serve_open(8, 63)
        tickets = {}
        for i in range(15):
            tickets[ctx.serve_submit("Edge", *inst[i])] = i
        steps = 0
        nxt = 15
        while True:
            st = ctx.serve_step(1)
            steps += 1
            if steps in (2, 5) or (steps > 5 and nxt < len(inst)):
                for i in range(nxt, min(nxt + 10, len(inst))):
                    tickets[ctx.serve_submit("Edge", *inst[i])] = i
                nxt = min(nxt + 10, len(inst))
            if st["active"] == 0 and st["pending"] == 0 and nxt == len(inst):
                break
            assert steps < 2000
        for t, i in tickets.items():
            assert ctx.serve_poll(t)
            c0, c1, counts = ctx.serve_result(t, "Reach")
            check(oracle.reach(*inst[i]), c0, c1, counts)
            ctx.serve_release(t)


@pytest.mark.parametrize("mode", [0, 1], ids=["matrix", "sorted"])
def test_serving_trickle_admissions(mode):
    """Two requests arrive per step into 8 slots: admission iterations run
    while retired instances still sit in their slots (their staged EDB
    tuples are derived again by the non-recursive rule and must be removed
    by their full), and slots are reused many times."""
    from paper_2311_02206_gb300 import hisa
    inst = instances(60, 7)
    with hisa.Context(flags=_full_modes()[mode]) as ctx:
        ctx.program(*oracle.REACH)
        ctx.serve_open(8, 63)
        tickets, nxt, retired = {}, 0, []
        for step in range(4000):
            for _ in range(2):
                if nxt < len(inst):
                    tickets[ctx.serve_submit("Edge", *inst[nxt])] = nxt
                    nxt += 1
            st = ctx.serve_step(1)
            got = ctx.serve_retired()   # what this step retired, no polling
            assert len(got) == st["retired"] and all(ctx.serve_poll(t) for t in got)
            retired += got
            if st["active"] == 0 and st["pending"] == 0 and nxt == len(inst):
                break
        assert sorted(retired) == sorted(tickets)
        for t, i in tickets.items():
            assert ctx.serve_poll(t)
            c0, c1, counts = ctx.serve_result(t, "Reach")
            check(oracle.reach(*inst[i]), c0, c1, counts)


def test_serving_budget_limits_admission():
    from paper_2311_02206_gb300 import hisa
    inst = [workloads.er_graph(40, 100, k) for k in range(6)]
    with hisa.Context() as ctx:
        ctx.program(*oracle.REACH)
        ctx.serve_open(16, 63, budget_bytes=1)      # at most one instance at a time
        tickets = [ctx.serve_submit("Edge", s, d) for s, d in inst]
        st = ctx.serve_step(1)
        assert st["admitted"] == 1 and st["pending"] == 5
        while st["active"] or st["pending"]:
            st = ctx.serve_step(4)
        for t, (s, d) in zip(tickets, inst):
            c0, c1, counts = ctx.serve_result(t, "Reach")
            check(oracle.reach(s, d), c0, c1, counts)


def test_batch_of_config_shapes():
    """Instances with the config's size law (log-uniform n, degree 1.5-4),
    scaled down to 64 instances with n <= 512."""
    from paper_2311_02206_gb300 import hisa
    specs = workloads.batch_instances(64, 4, n_lo_log2=6, n_hi_log2=9)
    graphs = [workloads.er_graph(n, m, sd) for n, m, sd in specs]
    with hisa.Context() as ctx:
        ctx.program(*oracle.REACH)
        for i, (s, d) in enumerate(graphs):
            ctx.load_instance("Edge", i, s, d)
        ctx.run()
        for i in range(0, 64, 7):
            c0, c1 = ctx.read_instance("Reach", i)
            check(oracle.reach(*graphs[i]), c0, c1, ctx.instance_delta_counts("Reach", i))


@pytest.mark.parametrize("knobs", [dict(radix_items=8), dict(load_factor=0.5), dict(dense_unit=64),
                                   dict(radix_items=16, dense_unit=1024, load_factor=0.65)])
def test_served_with_tuning_knobs(knobs):
    """The autotuner's knobs (sort tile, load factor of the hashed indexes,
    the grouped join's work split) change no result of a served batch."""
    from paper_2311_02206_gb300 import hisa
    inst = instances(24, 5, nmax=300)
    with hisa.Context(**knobs) as ctx:
        ctx.program(*oracle.REACH)
        ctx.serve_open(32, 300, 0)
        tickets = {ctx.serve_submit("Edge", s, d): i for i, (s, d) in enumerate(inst)}
        done = {}
        for _ in range(10000):
            ctx.serve_step(1)
            for t, i in list(tickets.items()):
                if i not in done and ctx.serve_poll(t):
                    done[i] = ctx.serve_result(t, "Reach")
                    ctx.serve_release(t)
            if len(done) == len(inst):
                break
        for i, (s, d) in enumerate(inst):
            c0, c1, dc = done[i]
            check(oracle.reach(s, d), c0, c1, dc)
