"""Helpers shared by the GPU parity tests: run a program through the C-ABI and
reduce GPU output for comparison with the oracle."""
from __future__ import annotations

import numpy as np

import oracle


def gpu_eval(relations, rules, edb, flags=None, **kw):
    """Evaluates a program with libhisa.so; returns (rels, counts, stats)."""
    from paper_2311_02206_gb300 import hisa
    if flags is None:
        flags = hisa.FLAG_GRAPH
    with hisa.Context(flags=flags, **kw) as ctx:
        ctx.program(relations, rules)
        for name, (c0, c1) in edb.items():
            ctx.load_tuples(name, c0, c1)
        st = ctx.run()
        rels, counts = {}, {}
        for name, kind in relations.items():
            if kind == "idb":
                rels[name] = ctx.read_relation(name)
                counts[name] = ctx.delta_counts(name)
        return rels, counts, st


def assert_same(rels_gpu, counts_gpu, ref: "oracle.Result"):
    for name, (c0, c1) in ref.relations.items():
        g0, g1 = rels_gpu[name]
        assert len(g0) == len(c0), (name, len(g0), len(c0))
        assert np.array_equal(g0, c0) and np.array_equal(g1, c1), name
        k = ref.iterations
        want = ref.delta_counts[name] + [0] * (k - len(ref.delta_counts[name]))
        assert counts_gpu[name] == want, (name, counts_gpu[name], want)


def fingerprint_device(c0, c1, chunk=1 << 27) -> int:
    """oracle.fingerprint of GPU tensors, reduced chunk by chunk on the host."""
    total = 0
    n = c0.numel()
    for s in range(0, n, chunk):
        a = c0[s:s + chunk].cpu().numpy().view(np.uint32)
        b = c1[s:s + chunk].cpu().numpy().view(np.uint32)
        total = (total + oracle.fingerprint(a, b)) % (1 << 64)
    return total


def assert_strictly_increasing_device(c0, c1, chunk=1 << 28):
    """The tuples (c0[i], c1[i]) of two int32 CUDA tensors (uint32 bit patterns)
    are in strictly increasing lexicographic order: every read must return a
    sorted set.  Checked on the device, chunk by chunk, over 64-bit codes."""
    import torch
    n = c0.numel()
    assert c1.numel() == n
    prev = None
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        code = ((c0[s:e].to(torch.int64) & 0xFFFFFFFF) << 32) | (c1[s:e].to(torch.int64) & 0xFFFFFFFF)
        # codes are below 2**64 as unsigned; flip the sign bit so signed order is unsigned order
        code = code ^ (-(1 << 63))
        if code.numel() > 1:
            assert bool((code[1:] > code[:-1]).all()), f"not strictly increasing in [{s}, {e})"
        if prev is not None and code.numel():
            assert int(code[0]) > prev, f"not strictly increasing at {s}"
        if code.numel():
            prev = int(code[-1])
        del code
