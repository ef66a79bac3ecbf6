"""CPU oracle for semi-naive Datalog evaluation and the HISA primitives.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the cpu-baseline / reference legs of ``bench.py``.  Nothing in the product
package imports it, and it imports nothing from the product package (only the
seeded input generators in ``paper_2311_02206_gb300.workloads`` and the
program texts in ``paper_2311_02206_gb300.programs``, which hold no
evaluation arithmetic).

* ``seminaive``  -- C++ std::set semi-naive evaluator (``seminaive.cpp``):
  Section 2 "Semi-naive evaluation" and Section 5.1 (join, populate delta,
  merge full/delta, clear new, repeat until delta is empty).
* ``naive``      -- a second, independent evaluator (pure Python sets) that
  iterates the immediate-consequence operator on the whole database; used
  only to pin the first one on tiny inputs.
* ``primitives`` -- plain definitions of the HISA building blocks (Section 4):
  sorted deduplicated data array, run index, set difference, merge, binary join.

A program is plain data: ``relations`` maps a name to ``"edb"`` or ``"idb"``;
``rules`` is a list of ``(head, body, neq)`` where ``head`` and each body atom
are ``(relation, (var, var))`` and ``neq`` lists ``(var, var)`` pairs that must
differ.  Variables are strings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "seminaive.cpp")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``seminaive.cpp`` into ``liboracle.so`` (plain g++, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, u32p, u64p, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), \
                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32)
            lib.oracle_new.restype = P
            lib.oracle_free.argtypes = [P]
            lib.oracle_add_relation.argtypes = [P, ctypes.c_int]
            lib.oracle_load.argtypes = [P, ctypes.c_int, u32p, u32p, ctypes.c_uint64]
            lib.oracle_add_rule.argtypes = [P, i32p, ctypes.c_int]
            lib.oracle_run.argtypes = [P, ctypes.c_uint32]
            lib.oracle_size.argtypes = [P, ctypes.c_int]
            lib.oracle_size.restype = ctypes.c_uint64
            lib.oracle_read.argtypes = [P, ctypes.c_int, u32p, u32p]
            lib.oracle_delta_counts.argtypes = [P, ctypes.c_int, u64p, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class Result:
    """Fixpoint of one program: sorted tuples and delta counts per IDB relation."""

    def __init__(self, relations, counts, iterations):
        self.relations = relations      # name -> (c0, c1) uint32 arrays, lexicographic
        self.delta_counts = counts      # name -> list[int], |delta_1| .. |delta_K|
        self.iterations = iterations    # K

    def size(self, name):
        return len(self.relations[name][0])


def seminaive(relations: dict, rules: list, edb: dict, max_iters: int = 1 << 20) -> Result:
    """Evaluate ``rules`` over the EDB tuples ``edb`` (name -> (c0, c1)) to the
    least fixpoint by semi-naive evaluation (Section 2; Section 5.1)."""
    lib = _load()
    h = lib.oracle_new()
    try:
        ids = {}
        for name, kind in relations.items():
            if kind not in ("edb", "idb"):
                raise ValueError(kind)
            ids[name] = lib.oracle_add_relation(h, 1 if kind == "idb" else 0)
        for name, (c0, c1) in edb.items():
            c0 = np.ascontiguousarray(c0, dtype=np.uint32)
            c1 = np.ascontiguousarray(c1, dtype=np.uint32)
            if lib.oracle_load(h, ids[name], _ptr(c0, ctypes.c_uint32), _ptr(c1, ctypes.c_uint32), len(c0)):
                raise RuntimeError("load failed")
        for head, body, neq in rules:
            names = {}

            def var(v):
                return names.setdefault(v, len(names))

            for b in body:          # variable ids in order of first use in the body
                var(b[1][0])
                var(b[1][1])
            desc = [ids[head[0]], var(head[1][0]), var(head[1][1]), len(body)]
            for b in body:
                desc += [ids[b[0]], var(b[1][0]), var(b[1][1])]
            desc.append(len(neq))
            for a, b in neq:
                desc += [var(a), var(b)]
            arr = np.array(desc, dtype=np.int32)
            rc = lib.oracle_add_rule(h, _ptr(arr, ctypes.c_int32), len(arr))
            if rc < 0:
                raise ValueError(f"bad rule {head} <- {body} (code {rc})")
        k = lib.oracle_run(h, max_iters)
        if k < 0:
            raise RuntimeError("oracle did not reach the fixpoint within max_iters")
        rels, counts = {}, {}
        for name, kind in relations.items():
            if kind != "idb":
                continue
            n = lib.oracle_size(h, ids[name])
            c0 = np.empty(n, np.uint32)
            c1 = np.empty(n, np.uint32)
            lib.oracle_read(h, ids[name], _ptr(c0, ctypes.c_uint32), _ptr(c1, ctypes.c_uint32))
            rels[name] = (c0, c1)
            buf = np.zeros(max(k, 1), np.uint64)
            got = lib.oracle_delta_counts(h, ids[name], _ptr(buf, ctypes.c_uint64), len(buf))
            counts[name] = [int(x) for x in buf[:got]]
        return Result(rels, counts, k)
    finally:
        lib.oracle_free(h)


# ---- programs used throughout ---------------------------------------------------------
# The Datalog programs are inputs, like the seeded EDB generators: plain data
# (relation kinds and rules) kept in a module of their own that both the
# oracle and the engine's callers read; it holds no evaluation arithmetic.
from paper_2311_02206_gb300.programs import CSPA, REACH, SG, SG_LITERAL  # noqa: E402,F401


def fingerprint(c0, c1) -> int:
    """Order-independent fingerprint of a binary relation: the sum modulo 2**64
    of the SplitMix64 finaliser of (c0 << 32 | c1) over its tuples."""
    x = (np.asarray(c0, np.uint64) << np.uint64(32)) | np.asarray(c1, np.uint64)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    x = x ^ (x >> np.uint64(31))
    return int(np.sum(x, dtype=np.uint64))


def reach(src, dst, **kw) -> Result:
    rels, rules = REACH
    return seminaive(rels, rules, {"Edge": (src, dst)}, **kw)


def reach_targets(src, dst, targets, **kw) -> Result:
    """REACH restricted to the target columns ``targets``.

    The recursive REACH rule keeps the ``to`` column of its Reach atom, so the
    tuples ending in a target set T are derived from Edge tuples ending in T
    alone: evaluating Reach(f,t) <- Edge(f,t), Tgt(t,t) together with the
    recursive rule gives exactly Reach restricted to V x T, and its delta at
    iteration k is delta_k restricted to V x T."""
    t = np.asarray(targets, dtype=np.uint32)
    rels = {"Edge": "edb", "Tgt": "edb", "Reach": "idb"}
    rules = [
        (("Reach", ("f", "t")), [("Edge", ("f", "t")), ("Tgt", ("t", "t"))], []),
        (("Reach", ("f", "t")), [("Edge", ("f", "m")), ("Reach", ("m", "t"))], []),
    ]
    return seminaive(rels, rules, {"Edge": (src, dst), "Tgt": (t, t)}, **kw)
