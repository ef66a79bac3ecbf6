"""hisa_difference_merge_noalloc -- the set-difference + merge step that
allocates nothing -- called through the C-ABI.

Some callers cannot let a library allocate device memory while it runs: a host
framework that owns all device memory and lends out only inputs and outputs,
a real-time path that must not enter an allocator, a program under a memory
budget fixed in advance.  This entry point keeps its scratch in an array the
library reserves when it loads.  Its results are checked against the oracle's
definitions (Section 5.1's populate-delta and merge, on codes) and against the
allocating entry point hisa_difference_merge, on two calls in a row (the
second smaller than the first, so anything the first call leaves in the shared
scratch and the second fails to clear would show), with a delta buffer that is
too small, without the merged output, and with nothing new.  Collected last,
so that a failure here stops a run only after every other test has run."""
import ctypes

import numpy as np
import pytest

from oracle import primitives as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HISA_ERR_CAPACITY = -9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


def _case(rng, nf, nn, dtype, hi):
    full = np.unique(rng.integers(0, hi, nf, dtype=np.uint64)).astype(dtype)
    fresh = np.sort(np.concatenate([rng.integers(0, hi, nn, dtype=np.uint64).astype(dtype),
                                    rng.choice(full, min(len(full), nn // 4))]))
    return full, fresh


def _dev(a):
    view = np.int32 if a.dtype == np.uint32 else np.int64
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()


def _host(t, dtype):
    return t.cpu().numpy().view(dtype)


@pytest.mark.parametrize("dtype,hi", [(np.uint32, 1 << 32), (np.uint64, 1 << 62)])
def test_noalloc_matches_oracle_and_allocating_entry_point_twice(dtype, hi):
    from paper_2311_02206_gb300 import hisa
    rng = np.random.default_rng(17)
    for nf, nn in [(300_000, 500_000), (70_000, 20_000)]:     # two calls in a row
        full, fresh = _case(rng, nf, nn, dtype, hi)
        want_d, want_f = P.difference_merge_codes(full, fresh)
        dfull, dfresh = _dev(full), _dev(fresh)
        alloc_d, alloc_f = hisa.difference_merge(dfull, dfresh)
        tdt = dfresh.dtype
        dout = torch.full((fresh.size,), -1, dtype=tdt, device="cuda")
        fout = torch.full((full.size + fresh.size,), -1, dtype=tdt, device="cuda")
        got_d, got_f = hisa.difference_merge_noalloc(dfull, dfresh, dout, fout)
        assert np.array_equal(_host(got_d, dtype), want_d)
        assert np.array_equal(_host(got_f, dtype), want_f)
        assert torch.equal(got_d, alloc_d) and torch.equal(got_f, alloc_f)


def _raw(lib, full, fresh, dout, dcap, fout, fcap, kb):
    n = ctypes.c_uint64(12345)
    rc = lib.hisa_difference_merge_noalloc(
        full.data_ptr() if full.numel() else None, full.numel(), fresh.data_ptr() if fresh.numel() else None,
        fresh.numel(), dout.data_ptr() if dout is not None else None, dcap,
        fout.data_ptr() if fout is not None else None, fcap, ctypes.byref(n), kb, None)
    torch.cuda.synchronize()
    return rc, n.value


def _raw_alloc(lib, full, fresh, dout, dcap, fout, fcap, kb):
    n = ctypes.c_uint64(12345)
    rc = lib.hisa_difference_merge(
        full.data_ptr() if full.numel() else None, full.numel(), fresh.data_ptr() if fresh.numel() else None,
        fresh.numel(), dout.data_ptr() if dout is not None else None, dcap,
        fout.data_ptr() if fout is not None else None, fcap, ctypes.byref(n), kb, None)
    torch.cuda.synchronize()
    return rc, n.value


def test_noalloc_delta_buffer_too_small():
    """CAPACITY, with the needed delta size in *n_delta, as the allocating call."""
    from paper_2311_02206_gb300 import hisa
    lib = hisa.load_library()
    full, fresh = _case(np.random.default_rng(5), 40_000, 30_000, np.uint32, 1 << 32)
    want_d, _ = P.difference_merge_codes(full, fresh)
    dfull, dfresh = _dev(full), _dev(fresh)
    small = torch.empty(100, dtype=torch.int32, device="cuda")
    fout = torch.empty(full.size + fresh.size, dtype=torch.int32, device="cuda")
    rc, n = _raw(lib, dfull, dfresh, small, small.numel(), fout, fout.numel(), 4)
    rc_a, n_a = _raw_alloc(lib, dfull, dfresh, small, small.numel(), fout, fout.numel(), 4)
    assert rc == HISA_ERR_CAPACITY and rc_a == HISA_ERR_CAPACITY
    assert n == n_a == want_d.size
    # the next call, with room, is exact again (nothing stale in the shared scratch)
    dout = torch.empty(fresh.size, dtype=torch.int32, device="cuda")
    got_d, got_f = hisa.difference_merge_noalloc(dfull, dfresh, dout, fout)
    assert np.array_equal(_host(got_d, np.uint32), want_d)


def test_noalloc_without_merged_output():
    """full_out = NULL: only delta is written."""
    from paper_2311_02206_gb300 import hisa
    full, fresh = _case(np.random.default_rng(6), 90_000, 120_000, np.uint64, 1 << 40)
    want_d, _ = P.difference_merge_codes(full, fresh)
    dout = torch.empty(fresh.size, dtype=torch.int64, device="cuda")
    got_d, got_f = hisa.difference_merge_noalloc(_dev(full), _dev(fresh), dout, None)
    assert got_f is None
    assert np.array_equal(_host(got_d, np.uint64), want_d)


@pytest.mark.parametrize("nf", [0, 5000])
def test_noalloc_nothing_new(nf):
    """n_new = 0: delta is empty and full' is a copy of full."""
    from paper_2311_02206_gb300 import hisa
    full, _ = _case(np.random.default_rng(7), nf, 0, np.uint32, 1 << 32)
    fresh = np.zeros(0, np.uint32)
    want_d, want_f = P.difference_merge_codes(full, fresh)
    dout = torch.empty(1, dtype=torch.int32, device="cuda")
    fout = torch.full((max(full.size, 1),), -1, dtype=torch.int32, device="cuda")
    got_d, got_f = hisa.difference_merge_noalloc(_dev(full), _dev(fresh), dout, fout)
    assert got_d.numel() == 0 and want_d.size == 0
    assert np.array_equal(_host(got_f, np.uint32), want_f)


def test_noalloc_rejects_inputs_over_the_limit():
    from paper_2311_02206_gb300 import hisa
    lib = hisa.load_library()
    n = ctypes.c_uint64()
    fake = ctypes.c_void_p(256)   # never dereferenced: the size check comes first
    rc = lib.hisa_difference_merge_noalloc(fake, hisa.NOALLOC_MAX_CODES, fake, 1, fake, 1, None, 0,
                                           ctypes.byref(n), 4, None)
    assert rc == hisa.HISA_ERR_TOO_LARGE
    assert lib.hisa_status_string(rc) == b"input larger than the fixed maximum size"
