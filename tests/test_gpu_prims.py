"""Kernel-level parity through the C-ABI primitives (include/hisa_prims.h)
against the oracle's definitions on codes, element by element, at sizes that
span several tiles plus a ragged tail, with the edge cases of each step."""
import numpy as np
import pytest

from oracle import primitives as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2311_02206_gb300 import build
    build.build()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


SIZES = [0, 1, 2, 31, 4095, 4096, 4097, 3 * 4096 + 17, 100_003, 1_048_576 + 333]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("bits", [8, 20, 32])
def test_sort_u32(n, bits):
    from paper_2311_02206_gb300 import hisa
    rng = np.random.default_rng(n * 7 + bits)
    x = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
    got = host(hisa.sort_codes(dev(x, np.int32), bits), np.uint32)
    assert np.array_equal(got, P.sort_codes(x))


@pytest.mark.parametrize("n", [0, 5, 3071, 3072, 3073, 250_001])
@pytest.mark.parametrize("bits", [33, 40, 64])
def test_sort_u64(n, bits):
    from paper_2311_02206_gb300 import hisa
    rng = np.random.default_rng(n + bits)
    x = rng.integers(0, 1 << 62, n, dtype=np.uint64)
    x = (x << np.uint64(2) | rng.integers(0, 4, n, dtype=np.uint64)) & np.uint64((1 << bits) - 1)
    got = host(hisa.sort_codes(dev(x, np.int64), bits), np.uint64)
    assert np.array_equal(got, P.sort_codes(x))


@pytest.mark.parametrize("case", ["all_equal", "max_key", "sorted", "reversed", "skewed"])
def test_sort_unique_edge_cases(case):
    from paper_2311_02206_gb300 import hisa
    n = 50_000
    rng = np.random.default_rng(1)
    if case == "all_equal":
        x = np.full(n, 7, np.uint32)
    elif case == "max_key":
        x = rng.integers(0xFFFFFF00, 0xFFFFFFFF, n, dtype=np.uint64, endpoint=True).astype(np.uint32)
    elif case == "sorted":
        x = np.arange(n, dtype=np.uint32) // 3
    elif case == "reversed":
        x = (np.arange(n, dtype=np.uint32) // 2)[::-1].copy()
    else:  # one hot digit, heavy repeats (R-MAT-like)
        x = np.where(rng.random(n) < 0.9, 0, rng.integers(0, 1 << 32, n, dtype=np.uint64)).astype(np.uint32)
    got = host(hisa.sort_unique_codes(dev(x, np.int32), 32), np.uint32)
    assert np.array_equal(got, P.sort_unique_codes(x))


def _sorted_unique(rng, n, hi, dtype):
    return np.unique(rng.integers(0, hi, n, dtype=np.uint64)).astype(dtype)


@pytest.mark.parametrize("nf,nn", [(0, 0), (0, 10), (10, 0), (5000, 5000), (70_000, 9_000), (9_000, 70_000),
                                   (200_001, 333_333)])
@pytest.mark.parametrize("width", [4, 8])
def test_difference_merge(nf, nn, width):
    from paper_2311_02206_gb300 import hisa
    dt, tdt = (np.uint32, np.int32) if width == 4 else (np.uint64, np.int64)
    rng = np.random.default_rng(nf + nn + width)
    hi = 3 * (nf + nn) + 10
    full = _sorted_unique(rng, nf, hi, dt)
    fresh = np.sort(np.concatenate([rng.integers(0, hi, nn, dtype=np.uint64).astype(dt),
                                    rng.choice(full, min(nn // 3, nf)) if nf else np.zeros(0, dt)]))
    fresh = np.sort(np.concatenate([fresh, fresh[: len(fresh) // 5]]))   # repeats, some spanning tiles
    d, f = hisa.difference_merge(dev(full, tdt), dev(fresh, tdt))
    wd, wf = P.difference_merge_codes(full, fresh)
    assert np.array_equal(host(d, dt), wd)
    assert np.array_equal(host(f, dt), wf)


def test_difference_merge_nothing_new_copies_full():
    from paper_2311_02206_gb300 import hisa
    full = np.arange(0, 30_000, 3, dtype=np.uint32)
    empty = np.zeros(0, np.uint32)
    for _ in range(2):
        junk = torch.full((full.size,), -1, dtype=torch.int32, device="cuda")   # dirty the allocator's cache
        del junk
        d, f = hisa.difference_merge(dev(full, np.int32), dev(empty, np.int32))
        assert d.numel() == 0 and np.array_equal(host(f, np.uint32), full)


def test_difference_merge_max_keys():
    from paper_2311_02206_gb300 import hisa
    full = np.array([0, 5, 0xFFFFFFFE, 0xFFFFFFFF], np.uint32)
    fresh = np.array([0, 0, 1, 0xFFFFFFFF, 0xFFFFFFFF], np.uint32)
    d, f = hisa.difference_merge(dev(full, np.int32), dev(fresh, np.int32))
    assert host(d, np.uint32).tolist() == [1]
    assert host(f, np.uint32).tolist() == [0, 1, 5, 0xFFFFFFFE, 0xFFFFFFFF]
    full64 = np.array([1, (1 << 64) - 1], np.uint64)
    fresh64 = np.array([(1 << 64) - 2, (1 << 64) - 1], np.uint64)
    d, f = hisa.difference_merge(dev(full64, np.int64), dev(fresh64, np.int64))
    assert host(d, np.uint64).tolist() == [(1 << 64) - 2]


@pytest.mark.parametrize("no,ni,dom", [(0, 10, 8), (10, 0, 8), (3000, 2000, 64), (40_000, 30_000, 1000),
                                       (5000, 60_000, 40)])
@pytest.mark.parametrize("proj", [(3, 1), (0, 3), (2, 1), (1, 0)])
def test_join(no, ni, dom, proj):
    from paper_2311_02206_gb300 import hisa
    b = 16
    rng = np.random.default_rng(no + ni + dom)
    outer = P.encode_rows(rng.integers(0, dom, (no, 2)), b, np.uint32)
    inner = np.unique(P.encode_rows(rng.integers(0, dom, (ni, 2)), b, np.uint32))
    for ocol in (0, 1):
        got = host(hisa.join_codes(dev(outer, np.int32), dev(inner, np.int32), b, ocol, *proj), np.uint32)
        want = P.join_codes(outer, inner, b, ocol, *proj, dtype=np.uint32)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("neq", [(1, 3), (3, 0), (0, 1), (2, 3)])
def test_join_with_filter(neq):
    from paper_2311_02206_gb300 import hisa
    b = 8
    rng = np.random.default_rng(sum(neq))
    outer = P.encode_rows(rng.integers(0, 20, (5000, 2)), b, np.uint32)
    inner = np.unique(P.encode_rows(rng.integers(0, 20, (300, 2)), b, np.uint32))
    code = 1 + 4 * neq[0] + neq[1]
    got = host(hisa.join_codes(dev(outer, np.int32), dev(inner, np.int32), b, 0, 1, 3, code), np.uint32)
    want = P.join_codes(outer, inner, b, 0, 1, 3, neq=neq, dtype=np.uint32)
    assert np.array_equal(got, want)


def test_join_skewed_hub():
    """One inner run of 20,000 tuples joined by many outer tuples: the write
    pass spreads the run over many chunks."""
    from paper_2311_02206_gb300 import hisa
    b = 16
    inner = P.encode_rows(np.stack([np.zeros(20_000, np.int64), np.arange(20_000)], 1), b, np.uint32)
    outer = P.encode_rows(np.stack([np.arange(300) % 3, np.arange(300)], 1), b, np.uint32)
    got = host(hisa.join_codes(dev(outer, np.int32), dev(inner, np.int32), b, 0, 3, 1), np.uint32)
    want = P.join_codes(outer, inner, b, 0, 3, 1, dtype=np.uint32)
    assert len(want) == 100 * 20_000
    assert np.array_equal(got, want)
