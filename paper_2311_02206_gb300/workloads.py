"""Seeded synthetic inputs for the semi-naive Datalog workloads.

This module only draws inputs; it holds none of the evaluation arithmetic, so
both the CPU oracle (``oracle/``) and the GPU path read their EDB relations
from here.  Every draw comes from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): value ``i`` of stream ``(seed, stream)`` is the SplitMix64
output mix of ``key + (i + 1) * 0x9E3779B97F4A7C15``.  Only integer
operations and IEEE basic float operations are used, so x86 and Arm hosts
produce the same bytes.

Graph shapes follow the paper's REACH / SG / CSPA workloads (Section 6): the
paper's SNAP, SuiteSparse, road-network and Graspan inputs are not available,
so synthetic graphs of the stated sizes and degree structure stand in.
"""
from __future__ import annotations

import math
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK32 = np.uint64(0xFFFFFFFF)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of one independent stream: the mix of ``seed`` and ``stream``."""
    k = np.array([(seed * 0x100000001B3 + stream * 0x51_7CC1_B727_220A_95) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _mix(k)[0]


def rand_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Values ``start .. start+count-1`` of stream ``(seed, stream)`` as uint64."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(key + idx * _GOLDEN)


def _below(r32: np.ndarray, n) -> np.ndarray:
    """Map 32-bit draws to [0, n) by multiply-shift (Lemire 2019)."""
    return ((r32 & _MASK32) * np.uint64(n)) >> np.uint64(32)


def _first_distinct(u: np.ndarray, v: np.ndarray, m: int, keep: np.ndarray):
    """First ``m`` distinct (u, v) pairs among those with ``keep`` set, in draw order."""
    u = u[keep]
    v = v[keep]
    code = (u.astype(np.uint64) << np.uint64(32)) | v.astype(np.uint64)
    _, first = np.unique(code, return_index=True)
    first.sort()
    return u[first[:m]], v[first[:m]], len(first)


def er_graph(n: int, m: int, seed: int, allow_self_loops: bool = False):
    """Directed G(n, m): uniform (u, v) draws, self-loops (unless allowed) and
    repeats rejected, until ``m`` distinct edges.  Returns (src, dst) uint32."""
    if m > n * n - (0 if allow_self_loops else n):
        raise ValueError("m exceeds the number of possible edges")
    drawn = 0
    batch = max(1024, 2 * m)
    us, vs = [], []
    while True:
        r = rand_u64(seed, 1, drawn, batch)
        drawn += batch
        us.append(_below(r, n))
        vs.append(_below(r >> np.uint64(32), n))
        u = np.concatenate(us)
        v = np.concatenate(vs)
        keep = np.ones(len(u), bool) if allow_self_loops else (u != v)
        a, b, got = _first_distinct(u, v, m, keep)
        if got >= m:
            return a.astype(np.uint32), b.astype(np.uint32)
        batch *= 2


# R-MAT quadrant thresholds as exact 32-bit fixed point: a=.57, a+b=.76, a+b+c=.95
_RMAT_T = (57 * (1 << 32) // 100, 76 * (1 << 32) // 100, 95 * (1 << 32) // 100)


def rmat_graph(scale: int, m: int, seed: int, return_draws: bool = False):
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with (a,b,c,d)=(.57,.19,.19,.05),
    no noise, no relabelling: each edge descends ``scale`` levels, one 32-bit
    draw per level picking a quadrant (row bit -> source, column bit -> target).
    Self-loops and repeats are dropped until ``m`` distinct edges remain."""
    t1, t2, t3 = (np.uint64(t) for t in _RMAT_T)
    words = (scale + 1) // 2
    drawn = 0
    batch = 2 * m
    us, vs = [], []
    while True:
        r = rand_u64(seed, 2, drawn * words, batch * words).reshape(batch, words)
        drawn += batch
        u = np.zeros(batch, np.uint64)
        v = np.zeros(batch, np.uint64)
        for lvl in range(scale):
            w = r[:, lvl // 2]
            x = (w >> np.uint64(32 * (lvl & 1))) & _MASK32
            q = (x >= t1).astype(np.uint64) + (x >= t2) + (x >= t3)
            bit = np.uint64(scale - 1 - lvl)
            u |= (q >> np.uint64(1)) << bit
            v |= (q & np.uint64(1)) << bit
        us.append(u)
        vs.append(v)
        ua = np.concatenate(us)
        va = np.concatenate(vs)
        a, b, got = _first_distinct(ua, va, m, ua != va)
        if got >= m:
            # raw draws consumed up to and including the m-th distinct edge
            res = (a.astype(np.uint32), b.astype(np.uint32))
            if return_draws:
                code = (ua.astype(np.uint64) << np.uint64(32)) | va
                keep = ua != va
                _, first = np.unique(code[keep], return_index=True)
                first.sort()
                kept_pos = np.nonzero(keep)[0][first[m - 1]]
                return res + (int(kept_pos) + 1,)
            return res
        batch *= 2


def dag_graph(n: int, m: int, max_gap: int, seed: int):
    """Random DAG: u uniform in [0, n), gap d uniform in [1, max_gap], v = u + d;
    draws with v >= n or repeats are rejected until ``m`` distinct edges."""
    drawn = 0
    batch = 2 * m
    us, vs = [], []
    while True:
        r = rand_u64(seed, 3, drawn, batch)
        drawn += batch
        u = _below(r, n)
        d = _below(r >> np.uint64(32), max_gap) + np.uint64(1)
        us.append(u)
        vs.append(u + d)
        ua = np.concatenate(us)
        va = np.concatenate(vs)
        a, b, got = _first_distinct(ua, va, m, va < np.uint64(n))
        if got >= m:
            return a.astype(np.uint32), b.astype(np.uint32)
        batch *= 2


# ---- closed-form shapes used by the pins --------------------------------------------

def path_graph(n: int):
    s = np.arange(n - 1, dtype=np.uint32)
    return s, s + 1


def cycle_graph(n: int):
    s = np.arange(n, dtype=np.uint32)
    return s, ((s + 1) % n).astype(np.uint32)


def complete_dag(n: int):
    u, v = np.triu_indices(n, k=1)
    return u.astype(np.uint32), v.astype(np.uint32)


def binary_tree(depth: int):
    """Complete binary tree with levels 0..depth; node i has children 2i+1, 2i+2."""
    nodes = (1 << (depth + 1)) - 1
    child = np.arange(1, nodes, dtype=np.uint32)
    return ((child - 1) // 2).astype(np.uint32), child


# ---- the five workload shapes ---------------------------------------------------------

def _exp2(x: float) -> float:
    """2**x from IEEE basic operations only (Taylor series of e**(f ln 2) on the
    fractional part), so every host gets the same double."""
    k = math.floor(x)
    f = (x - k) * 0.6931471805599453
    term, s = 1.0, 1.0
    for i in range(1, 30):
        term = term * f / i
        s = s + term
    return s * float(1 << k) if k >= 0 else s / float(1 << -k)


def batch_instances(count: int, seed: int, n_lo_log2: int = 6, n_hi_log2: int = 13,
                    deg_lo: float = 1.5, deg_hi: float = 4.0):
    """Sizes of independent REACH instances: node count log-uniform in
    [2**n_lo_log2, 2**n_hi_log2], mean out-degree uniform in [deg_lo, deg_hi],
    m = round(n * deg) distinct ER edges.  Returns a list of (n, m, edge_seed)."""
    r = rand_u64(seed, 5, 0, 2 * count)
    out = []
    for i in range(count):
        u1 = float(int(r[2 * i] >> np.uint64(11))) / float(1 << 53)
        u2 = float(int(r[2 * i + 1] >> np.uint64(11))) / float(1 << 53)
        n = int(round(_exp2(n_lo_log2 + (n_hi_log2 - n_lo_log2) * u1)))
        deg = deg_lo + (deg_hi - deg_lo) * u2
        m = int(round(n * deg))
        m = min(m, n * (n - 1))
        out.append((n, m, seed * 1_000_003 + i))
    return out


# ---- Zipf draws with IEEE basic operations only ------------------------------------------

_LN2 = 0.6931471805599453


def _ln(x: np.ndarray) -> np.ndarray:
    """Natural log of positive doubles: frexp range reduction and the atanh
    series 2 (t + t^3/3 + ...) with t = (m - 1) / (m + 1), m in [sqrt(1/2), sqrt(2))."""
    m, e = np.frexp(np.asarray(x, np.float64))
    small = m < 0.7071067811865476
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    acc = np.zeros_like(t)
    for k in range(41, 0, -2):
        acc = acc * t2 + 1.0 / k
    return 2.0 * t * acc + e * _LN2


def _exp(x: np.ndarray) -> np.ndarray:
    """e**x for moderate x: x = k ln2 + r, |r| <= ln2/2, Taylor series of e**r."""
    x = np.asarray(x, np.float64)
    k = np.floor(x / _LN2 + 0.5)
    r = x - k * _LN2
    acc = np.ones_like(r)
    term = np.ones_like(r)
    for i in range(1, 24):
        term = term * r / i
        acc = acc + term
    return np.ldexp(acc, k.astype(np.int64))


def zipf_ranks(count: int, n: int, s: float, seed: int, stream: int) -> np.ndarray:
    """Ranks 0..n-1 with P(rank k) proportional to (k+1)**-s, by inverse CDF
    of uniform 53-bit draws over the exact (IEEE basic-operation) CDF table."""
    w = _exp(-s * _ln(np.arange(1, n + 1, dtype=np.float64)))
    cdf = np.cumsum(w)
    u = (rand_u64(seed, stream, 0, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return np.minimum(np.searchsorted(cdf, u * cdf[-1], side="right"), n - 1).astype(np.int64)


def cspa_inputs(n_assign: int = 400_000, n_deref: int = 200_000, ids: int = 300_000, window: int = 1024,
                p_window: float = 0.8, s: float = 1.1, seed: int = 2):
    """Assign and Dereference pairs over ids [0, ids): the first id is Zipf(s)
    (rank - 1), the second with probability p_window uniform in the same
    aligned window of `window` ids, else Zipf(s); self-pairs and repeats are
    dropped until the requested number of distinct pairs."""
    out = []
    for rel, (count, stream) in enumerate([(n_assign, 10), (n_deref, 20)]):
        pairs_a, pairs_b = np.zeros(0, np.int64), np.zeros(0, np.int64)
        drawn, batch = 0, 2 * count
        while True:
            a = zipf_ranks(batch, ids, s, seed + drawn, stream)
            z = zipf_ranks(batch, ids, s, seed + drawn, stream + 1)
            r = rand_u64(seed + drawn, stream + 2, 0, batch)
            inwin = (r >> np.uint64(11)).astype(np.float64) / float(1 << 53) < p_window
            off = (((r & _MASK32) * np.uint64(window)) >> np.uint64(32)).astype(np.int64)
            b = np.where(inwin, np.minimum((a // window) * window + off, ids - 1), z)
            pairs_a = np.concatenate([pairs_a, a])
            pairs_b = np.concatenate([pairs_b, b])
            x, y, got = _first_distinct(pairs_a.astype(np.uint64), pairs_b.astype(np.uint64), count,
                                        pairs_a != pairs_b)
            drawn += 1
            if got >= count:
                out.append((x.astype(np.uint32), y.astype(np.uint32)))
                break
    return {"Assign": out[0], "Dereference": out[1]}


def config_reach_er(seed: int = 0):
    """REACH on ER n=1,000, m=3,000 (the small single-instance case)."""
    return er_graph(1000, 3000, seed)


def config_reach_rmat(seed: int = 3):
    """REACH on R-MAT scale 16 (65,536 nodes) with 2**19 distinct edges."""
    return rmat_graph(16, 1 << 19, seed)


def config_cspa(div: int = 250, window: int = 128, seed: int = 2):
    """The points-to inputs (Assign 400k, Dereference 200k, 300k ids, Zipf 1.1,
    80% in-window pairs) with the three counts divided by `div`.  The undivided
    counts derive far more than a GPU holds (see the design notes); 1/250 with
    windows of 128 ids derives ~4.6e9 raw tuples over ten iterations."""
    return cspa_inputs(400_000 // div, 200_000 // div, 300_000 // div, window=window, seed=seed)


def config_sg_dag(seed: int = 1):
    """SG on a random DAG with 20,000 nodes and 40,000 edges, gaps in [1, 256]."""
    return dag_graph(20000, 40000, 256, seed)
