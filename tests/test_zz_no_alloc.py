"""hisa_difference_merge_noalloc -- the variant of the set-difference + merge
step that allocates nothing -- against hisa_difference_merge, called through
the C-ABI.  Some callers cannot allocate device memory while they run (an
allocation-free stream capture, a real-time path, a fixed memory budget); this
entry point keeps its scratch in an array reserved when the library loads.
Two calls in a row, the second smaller than the first, so anything the first
call leaves in the shared scratch and the second fails to clear would show."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


def _case(rng, nf, nn, dtype, hi):
    full = np.unique(rng.integers(0, hi, nf, dtype=np.uint64)).astype(dtype)
    fresh = np.sort(np.concatenate([rng.integers(0, hi, nn, dtype=np.uint64).astype(dtype),
                                    rng.choice(full, min(len(full), nn // 4))]))
    tdt = torch.int32 if dtype == np.uint32 else torch.int64
    view = np.int32 if dtype == np.uint32 else np.int64
    return (torch.from_numpy(full.view(view)).cuda(), torch.from_numpy(fresh.view(view)).cuda(), tdt)


@pytest.mark.parametrize("dtype,hi", [(np.uint32, 1 << 32), (np.uint64, 1 << 62)])
def test_noalloc_matches_allocating_entry_point_twice(dtype, hi):
    from paper_2311_02206_gb300 import hisa
    rng = np.random.default_rng(17)
    for nf, nn in [(300_000, 500_000), (70_000, 20_000)]:     # two calls in a row
        full, fresh, tdt = _case(rng, nf, nn, dtype, hi)
        want_d, want_f = hisa.difference_merge(full, fresh)
        dout = torch.full((fresh.numel(),), -1, dtype=tdt, device="cuda")
        fout = torch.full((full.numel() + fresh.numel(),), -1, dtype=tdt, device="cuda")
        got_d, got_f = hisa.difference_merge_noalloc(full, fresh, dout, fout)
        assert torch.equal(got_d, want_d)
        assert torch.equal(got_f, want_f)


def test_noalloc_rejects_inputs_over_the_limit():
    from paper_2311_02206_gb300 import hisa
    import ctypes
    lib = hisa.load_library()
    n = ctypes.c_uint64()
    fake = ctypes.c_void_p(256)   # never dereferenced: the size check comes first
    rc = lib.hisa_difference_merge_noalloc(fake, hisa.NOALLOC_MAX_CODES, fake, 1, fake, 1, None, 0,
                                           ctypes.byref(n), 4, None)
    assert rc == hisa.HISA_ERR_TOO_LARGE
    assert lib.hisa_status_string(rc) == b"input larger than the fixed maximum size"
