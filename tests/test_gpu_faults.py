"""Failure paths, made to happen without faulting the GPU:

* every bounded device-side wait (decoupled look-back over earlier tiles,
  the mbarrier of a radix pass's tile copy) runs out on a word that nothing
  publishes, the kernel returns and the call reports HISA_ERR_DEVICE_TIMEOUT;
  the stream stays usable;
* an allocator hook that refuses the N-th allocation makes the call fail
  with HISA_ERR_OOM, and the same context then evaluates the program exactly;
* the read scratch that a read into page-locked host columns keeps gives way
  when a later run within the HBM budget needs the memory.

The paper describes no failure handling; these are the library's own
guarantees (include/hisa.h: no call traps or aborts)."""
import numpy as np
import pytest

import oracle
from paper_2311_02206_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HISA_ERR_OOM = -3
HISA_ERR_DEVICE_TIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_bounded_wait_runs_out_and_returns(which):
    from paper_2311_02206_gb300 import hisa
    assert hisa.check_bounded_wait(which, 64) == HISA_ERR_DEVICE_TIMEOUT
    # the stream and the context are still usable: an exact sort right after
    keys = torch.randint(0, 1 << 31, (100_000,), dtype=torch.int64, device="cuda").to(torch.int32)
    got = hisa.sort_codes(keys, 32)
    want = np.sort(keys.cpu().numpy().view(np.uint32))
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want)


def test_bounded_wait_argument_checks():
    from paper_2311_02206_gb300 import hisa
    assert hisa.check_bounded_wait(4, 64) == -1
    assert hisa.check_bounded_wait(0, 0) == -1
    assert hisa.check_bounded_wait(0, 1 << 20) == -1


class FailingAllocator:
    """torch's caching allocator that refuses the allocation numbered `fail_at`
    (1-based, counted after the context is created; 0 = never)."""

    def __init__(self, device=0):
        self.device = device
        self.calls = 0
        self.fail_at = 0
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at and self.calls == self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(nbytes, self.device, stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes, stream):
        self.live.pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)


def _evaluate(ctx, program, edb):
    for name, (c0, c1) in edb.items():
        ctx.load_tuples(name, c0, c1)
    ctx.run()
    return {name: ctx.read_relation(name) for name, kind in program[0].items() if kind == "idb"}


@pytest.mark.parametrize("prog", ["reach", "sg"])
def test_failed_allocation_reports_oom_and_context_recovers(prog):
    from paper_2311_02206_gb300 import hisa
    if prog == "reach":
        program, edb = oracle.REACH, {"Edge": workloads.er_graph(300, 900, 5)}
    else:
        program, edb = oracle.SG, {"Edge": workloads.dag_graph(200, 500, 16, 2)}
    ref = oracle.seminaive(*program, edb)
    # how many allocations one context makes through a load, a run and the reads
    counter = FailingAllocator()
    with hisa.Context(allocator=(counter.alloc, counter.free)) as ctx:
        counter.calls = 0
        ctx.program(*program)
        _evaluate(ctx, program, edb)
        total = counter.calls
    assert total > 5
    failures = 0
    for n in sorted(set(np.linspace(1, total, min(total, 24)).astype(int).tolist())):
        fa = FailingAllocator()
        with hisa.Context(allocator=(fa.alloc, fa.free)) as ctx:
            ctx.program(*program)
            fa.calls = 0
            fa.fail_at = n
            try:
                got = _evaluate(ctx, program, edb)
            except hisa.HisaError as e:
                assert e.status == HISA_ERR_OOM, (n, e)
                failures += 1
                fa.fail_at = 0
                ctx.reset_edb()
                got = _evaluate(ctx, program, edb)   # the same context, allocations allowed again
            for name, (w0, w1) in ref.relations.items():
                g0, g1 = got[name]
                assert np.array_equal(g0, w0) and np.array_equal(g1, w1), (n, name)
        assert not fa.live, "library-owned memory left after destroy"
    assert failures > 0


def test_run_after_pinned_read_within_budget():
    """A read into page-locked host columns keeps its device staging columns
    and bit matrix for the next read.  A later, larger run within an HBM
    budget equal to the peak of the same sequence with device reads (which
    keep no staging) must still succeed: the kept read scratch is released
    when an allocation would pass the budget."""
    from paper_2311_02206_gb300 import hisa
    small = workloads.config_reach_er()
    big = workloads.er_graph(2500, 9000, 3)
    ref = oracle.reach(*small)
    w0, w1 = ref.relations["Reach"]
    with hisa.Context() as ctx:
        ctx.program(*oracle.REACH)
        ctx.load_tuples("Edge", *small)
        ctx.run()
        ctx.read_relation("Reach", device=True)
        ctx.reset_edb()
        ctx.load_tuples("Edge", *big)
        ctx.run()
        b0, b1 = ctx.read_relation("Reach", device=True)
        b0, b1 = b0.cpu().numpy(), b1.cpu().numpy()
        peak = ctx.run().peak_bytes   # the context's high-water mark, the reads included
    n = len(w0)
    h0 = torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    h1 = torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    with hisa.Context(hbm_budget_bytes=peak) as ctx:
        ctx.program(*oracle.REACH)
        ctx.load_tuples("Edge", *small)
        ctx.run()
        g0, g1 = ctx.read_relation("Reach", out=(h0, h1))
        assert np.array_equal(g0, w0) and np.array_equal(g1, w1)
        ctx.reset_edb()
        ctx.load_tuples("Edge", *big)
        ctx.run()
        c0, c1 = ctx.read_relation("Reach", device=True)
        assert np.array_equal(c0.cpu().numpy(), b0) and np.array_equal(c1.cpu().numpy(), b1)
