"""Pins of the CPU oracle against facts it does not compute itself: brute-force
BFS closure and shortest-path counts, closed forms, a second independent
evaluator (naive iteration), the paper's worked examples, and planted mistakes
that these pins must catch."""
import os
import subprocess
import ctypes
from collections import deque

import numpy as np
import pytest

import oracle
from oracle import naive, primitives
from paper_2311_02206_gb300 import workloads
from programs import PROGRAMS, TC_NONLINEAR


# ---- REACH against BFS ---------------------------------------------------------------

def bfs_reach(n, src, dst):
    """All-pairs shortest path lengths >= 1 by BFS (dist(u, u) = shortest cycle).
    Returns dict (u, v) -> length."""
    adj = [[] for _ in range(n)]
    for a, b in zip(src.tolist(), dst.tolist()):
        adj[a].append(b)
    out = {}
    for u in range(n):
        dist = {}
        q = deque()
        for v in adj[u]:
            if v not in dist:
                dist[v] = 1
                q.append(v)
        while q:
            x = q.popleft()
            for y in adj[x]:
                if y not in dist:
                    dist[y] = dist[x] + 1
                    q.append(y)
        for v, dd in dist.items():
            out[(u, v)] = dd
    return out


def counts_from_dist(dist):
    if not dist:
        return []
    k = max(dist.values())
    c = [0] * k
    for dd in dist.values():
        c[dd - 1] += 1
    return c


@pytest.mark.parametrize("seed", range(120))
def test_reach_equals_bfs_closure(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    loops = bool(seed % 3 == 0)
    m = int(rng.integers(0, min(3 * n, n * n - (0 if loops else n)) + 1))
    src, dst = workloads.er_graph(n, m, seed, allow_self_loops=loops) if m else \
        (np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    r = oracle.reach(src, dst)
    dist = bfs_reach(n, src, dst)
    got = set(zip(*(x.tolist() for x in r.relations["Reach"])))
    assert got == set(dist)
    assert r.delta_counts["Reach"] == counts_from_dist(dist)


def test_reach_config_small_er_equals_bfs():
    src, dst = workloads.config_reach_er()
    r = oracle.reach(src, dst)
    dist = bfs_reach(1000, src, dst)
    assert r.size("Reach") == len(dist)
    assert r.delta_counts["Reach"] == counts_from_dist(dist)
    c0, c1 = r.relations["Reach"]
    assert set(zip(c0.tolist(), c1.tolist())) == set(dist)


# ---- closed forms --------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 10, 33])
def test_reach_path(n):
    r = oracle.reach(*workloads.path_graph(n))
    assert r.size("Reach") == n * (n - 1) // 2
    assert r.delta_counts["Reach"] == [n - k for k in range(1, n)]


@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_reach_cycle(n):
    r = oracle.reach(*workloads.cycle_graph(n))
    assert r.size("Reach") == n * n
    assert r.delta_counts["Reach"] == [n] * n


@pytest.mark.parametrize("n", [2, 6, 25])
def test_reach_complete_dag(n):
    r = oracle.reach(*workloads.complete_dag(n))
    c0, c1 = r.relations["Reach"]
    assert r.size("Reach") == n * (n - 1) // 2
    assert np.all(c0 < c1)
    assert r.delta_counts["Reach"] == [n * (n - 1) // 2]


@pytest.mark.parametrize("depth", [1, 2, 3, 5])
def test_sg_binary_tree_closed_form(depth):
    """SG on a complete binary tree: all ordered pairs of distinct nodes at the
    same depth; the pairs whose lowest common ancestor is k levels up appear in
    iteration k, 2**d * 2**(k-1) of them at depth d >= k."""
    r = oracle.seminaive(*oracle.SG, {"Edge": workloads.binary_tree(depth)})
    assert r.size("SG") == sum((1 << d) * ((1 << d) - 1) for d in range(1, depth + 1))
    expect = [sum((1 << d) << (k - 1) for d in range(k, depth + 1)) for k in range(1, depth + 1)]
    assert r.delta_counts["SG"] == expect


# ---- second evaluator ----------------------------------------------------------------

def _tiny_graph(seed, n=9, m=14):
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    return s, d


@pytest.mark.parametrize("name", sorted(PROGRAMS))
@pytest.mark.parametrize("seed", range(12))
def test_seminaive_equals_naive(name, seed):
    rels, rules = PROGRAMS[name]
    edb_names = [k for k, v in rels.items() if v == "edb"]
    edb = {e: _tiny_graph(seed * 7 + i) for i, e in enumerate(edb_names)}
    r = oracle.seminaive(rels, rules, edb)
    want, counts = naive.naive(rels, rules, edb)
    for n in want:
        got = list(zip(*(x.tolist() for x in r.relations[n])))
        assert got == want[n], n
    # delta counts: naive round k finds exactly delta_k (lists padded to K)
    k = max(len(c) for c in counts.values())
    for n in counts:
        assert r.delta_counts[n] == counts[n] + [0] * (k - len(counts[n])), n


@pytest.mark.parametrize("seed", range(8))
def test_cspa_seminaive_equals_naive(seed):
    """The ten-rule points-to program (three IDB relations in mutual
    recursion, two three-atom rules) on tiny skewed inputs."""
    edb = workloads.cspa_inputs(25 + seed, 12, 14, window=4, seed=seed)
    r = oracle.seminaive(*oracle.CSPA, edb)
    want, counts = naive.naive(*oracle.CSPA, edb)
    for n in want:
        assert list(zip(*(x.tolist() for x in r.relations[n]))) == want[n], n
    k = max(len(c) for c in counts.values())
    for n in counts:
        assert r.delta_counts[n] == counts[n] + [0] * (k - len(counts[n])), n


def doubling_counts(n_pairs_at, longest):
    """|delta_k| of the non-linear closure when the pairs at shortest distance
    l number n_pairs_at(l): iteration 1 finds l = 1, iteration k >= 2 the
    lengths in (2**(k-2), 2**(k-1)] (paths of both halves are already known)."""
    out = [n_pairs_at(1)]
    k = 2
    while (1 << (k - 2)) < longest:
        out.append(sum(n_pairs_at(l) for l in range((1 << (k - 2)) + 1, min(1 << (k - 1), longest) + 1)))
        k += 1
    return out


@pytest.mark.parametrize("n", [2, 3, 17, 64, 100])
def test_tc_nonlinear_path_closed_form(n):
    r = oracle.seminaive(*TC_NONLINEAR, {"E": workloads.path_graph(n)})
    assert r.size("T") == n * (n - 1) // 2
    assert r.delta_counts["T"] == doubling_counts(lambda l: n - l, n - 1)


@pytest.mark.parametrize("n", [1, 5, 32, 33])
def test_tc_nonlinear_cycle_closed_form(n):
    r = oracle.seminaive(*TC_NONLINEAR, {"E": workloads.cycle_graph(n)})
    assert r.size("T") == n * n
    assert r.delta_counts["T"] == doubling_counts(lambda l: n, n)


# ---- the paper's worked examples -----------------------------------------------------

def test_sg_example_narrative():
    """Section 2 example: SG(7,8) from Edge(4,7), Edge(4,8) in iteration 1;
    SG(6,8) from Edge(3,6), SG(3,4), Edge(4,8) in iteration 2; the third
    iteration finds nothing new (with a common parent 1 of 3 and 4)."""
    src = np.array([1, 1, 4, 4, 3], np.uint32)
    dst = np.array([3, 4, 7, 8, 6], np.uint32)
    rels, rules = oracle.SG
    want, counts = naive.naive(rels, rules, {"Edge": (src, dst)})
    r = oracle.seminaive(rels, rules, {"Edge": (src, dst)})
    got = set(zip(*(x.tolist() for x in r.relations["SG"])))
    assert (7, 8) in got and (6, 8) in got and (3, 4) in got
    assert r.delta_counts["SG"] == [4, 4]      # iteration 3 is empty: the fixpoint
    # (7,8) is already in delta_1; (6,8) first appears in delta_2
    r1 = oracle.seminaive(rels, [rules[0]], {"Edge": (src, dst)})
    assert (7, 8) in set(zip(*(x.tolist() for x in r1.relations["SG"])))
    assert (6, 8) not in set(zip(*(x.tolist() for x in r1.relations["SG"])))


def test_sorted_index_array_example():
    """Section 4.2: tuples {2,1,5}, {2,5,9}, {2,1,2} with the second column as
    join column reorder to (1,2,5), (5,2,9), (1,2,2) and sort as
    (1,2,2) < (1,2,5) < (5,2,9).  (The permutation printed beside the example
    reads 1,0,2; the stated order gives positions 2,0,1.)"""
    rows = np.array([[2, 1, 5], [2, 5, 9], [2, 1, 2]], np.uint32)
    idx = primitives.sorted_index_array(rows, [1])
    r = primitives.reorder_columns(rows, [1])
    assert r[idx].tolist() == [[1, 2, 2], [1, 2, 5], [5, 2, 9]]
    assert idx.tolist() == [2, 0, 1]


def test_foobar_join_example():
    """Section 5.1: Foo(2,3,5), Foo(2,3,2) joined with Bar(2,3,1) on the first
    two columns gives Foobar(5,1) and Foobar(2,1)."""
    foo = np.array([[2, 3, 5], [2, 3, 2]], np.uint32)
    bar = np.array([[2, 3, 1]], np.uint32)
    out = primitives.join(foo, [0, 1], bar, [0, 1], [("o", 2), ("i", 2)])
    assert out.tolist() == [[5, 1], [2, 1]]


# ---- primitives against brute force --------------------------------------------------

@pytest.mark.parametrize("seed", range(20))
def test_primitives_brute_force(seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 4, (int(rng.integers(0, 30)), 2)).astype(np.uint32)
    b = rng.integers(0, 4, (int(rng.integers(0, 30)), 2)).astype(np.uint32)
    sa, sb = sorted(set(map(tuple, a.tolist()))), sorted(set(map(tuple, b.tolist())))
    assert [tuple(x) for x in primitives.sort_unique(a).tolist()] == sa
    assert [tuple(x) for x in primitives.set_difference(a, primitives.sort_unique(b)).tolist()] == \
        sorted(set(sa) - set(sb))
    delta = sorted(set(sa) - set(sb))
    assert [tuple(x) for x in primitives.merge(np.array(sb, np.uint32).reshape(-1, 2),
                                               np.array(delta, np.uint32).reshape(-1, 2)).tolist()] == \
        sorted(set(sb) | set(delta))
    keys, begin, length = primitives.run_index(np.array(sa, np.uint32).reshape(-1, 2), 1)
    for k, bg, ln in zip(keys[:, 0].tolist(), begin.tolist(), length.tolist()):
        pos = [i for i, t in enumerate(sa) if t[0] == k]
        assert pos == list(range(bg, bg + ln))
    j = primitives.join(a, [1], b, [0], [("o", 0), ("i", 1)])
    brute = [(x[0], y[1]) for x in a.tolist() for y in b.tolist() if x[1] == y[0]]
    assert [tuple(x) for x in j.tolist()] == brute


def test_reach_targets_is_restriction():
    for seed in range(10):
        s, d = _tiny_graph(seed, n=12, m=30)
        full = oracle.reach(s, d)
        T = np.array([1, 4, 7, 11], np.uint32)
        part = oracle.reach_targets(s, d, T)
        c0, c1 = full.relations["Reach"]
        keep = np.isin(c1, T)
        assert np.array_equal(part.relations["Reach"][0], c0[keep])
        assert np.array_equal(part.relations["Reach"][1], c1[keep])
        dist = bfs_reach(12, s, d)
        sub = {k: v for k, v in dist.items() if k[1] in set(T.tolist())}
        assert part.delta_counts["Reach"] == counts_from_dist(sub)


def test_fingerprint_is_order_independent():
    s, d = _tiny_graph(3, n=50, m=100)
    p = np.random.default_rng(0).permutation(len(s))
    assert oracle.fingerprint(s, d) == oracle.fingerprint(s[p], d[p])
    assert oracle.fingerprint(s, d) != oracle.fingerprint(d, s)


# ---- planted mistakes: each must fail one of the pins above --------------------------

def _planted(k, tmp_path):
    so = str(tmp_path / f"liboracle_plant{k}.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", f"-DORACLE_PLANT={k}",
                           os.path.join(os.path.dirname(oracle.__file__), "seminaive.cpp"), "-o", so])
    return so


def _pins_pass():
    """A compact run of the pins; False as soon as one fails."""
    try:
        for n in (5, 9):
            r = oracle.reach(*workloads.path_graph(n))
            if r.size("Reach") != n * (n - 1) // 2 or r.delta_counts["Reach"] != [n - k for k in range(1, n)]:
                return False
            r = oracle.reach(*workloads.cycle_graph(n), max_iters=64)
            if r.size("Reach") != n * n or r.delta_counts["Reach"] != [n] * n:
                return False
        s, d = workloads.er_graph(12, 20, 5)
        r = oracle.reach(s, d)
        if set(zip(*(x.tolist() for x in r.relations["Reach"]))) != set(bfs_reach(12, s, d)):
            return False
        r = oracle.seminaive(*oracle.SG, {"Edge": workloads.binary_tree(3)})
        if r.size("SG") != 2 * 1 + 4 * 3 + 8 * 7:
            return False
        for name in ("tc_nonlinear", "mutual"):
            rels, rules = PROGRAMS[name]
            edb_names = [k for k, v in rels.items() if v == "edb"]
            for seed in range(6):
                edb = {e: _tiny_graph(seed * 7 + i) for i, e in enumerate(edb_names)}
                want, counts = naive.naive(rels, rules, edb)
                r = oracle.seminaive(rels, rules, edb)
                k = max(len(c) for c in counts.values())
                for n in want:
                    if list(zip(*(x.tolist() for x in r.relations[n]))) != want[n] or \
                            r.delta_counts[n] != counts[n] + [0] * (k - len(counts[n])):
                        return False
        return True
    except RuntimeError:
        return False


def test_pins_pass_on_the_oracle():
    assert _pins_pass()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_pins_catch_planted_mistake(k, tmp_path, monkeypatch):
    so = _planted(k, tmp_path)
    lib = ctypes.CDLL(so)
    saved = oracle._lib
    try:
        oracle._lib = None
        monkeypatch.setattr(oracle, "build", lambda force=False: so)
        oracle._load()
        assert not _pins_pass(), f"planted mistake {k} went unnoticed"
    finally:
        oracle._lib = saved
    del lib


def test_code_join_matches_tuple_join():
    """The code-level join definition agrees with the nested-loop definition."""
    rng = np.random.default_rng(5)
    b = 6
    o = rng.integers(0, 9, (60, 2)).astype(np.uint32)
    i = np.unique(rng.integers(0, 9, (40, 2)).astype(np.uint32), axis=0)
    for col in (0, 1):
        for proj in [(3, 1), (0, 2), (1, 3)]:
            side = [("o", 0), ("o", 1), ("i", 0), ("i", 1)]
            want = primitives.join(o, [col], i, [0], [side[proj[0]], side[proj[1]]])
            got = primitives.join_codes(primitives.encode_rows(o, b), primitives.encode_rows(i, b), b, col, *proj)
            assert np.array_equal(primitives.decode_codes(got, b), want)
    got = primitives.join_codes(primitives.encode_rows(o, b), primitives.encode_rows(i, b), b, 0, 1, 3, neq=(1, 3))
    want = [(x[1], y[1]) for x in o.tolist() for y in i.tolist() if x[0] == y[0] and x[1] != y[1]]
    assert [tuple(r) for r in primitives.decode_codes(got, b).tolist()] == want


def test_code_difference_merge_brute_force():
    rng = np.random.default_rng(9)
    full = np.unique(rng.integers(0, 50, 30)).astype(np.uint64)
    fresh = np.sort(rng.integers(0, 50, 40)).astype(np.uint64)
    d, f = primitives.difference_merge_codes(full, fresh)
    assert d.tolist() == sorted(set(fresh.tolist()) - set(full.tolist()))
    assert f.tolist() == sorted(set(full.tolist()) | set(fresh.tolist()))
