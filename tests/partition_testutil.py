"""Per-partition steps of the partitioned REACH written with the oracle's
definitions on torch CPU tensors, so that the iteration and exchange logic of
paper_2311_02206_gb300.partitioned runs on CPU ranks (gloo) without a GPU."""
from __future__ import annotations

import numpy as np
import torch

from oracle import primitives as P


def fmix32(x):
    """MurmurHash3's 32-bit finaliser (Appleby), elementwise on uint32."""
    h = np.asarray(x, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    m = np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & m
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & m
    h ^= h >> np.uint64(16)
    return h


def owner(values, nparts):
    return (fmix32(values) % np.uint64(nparts)).astype(np.int64)


def _np(t):
    return t.numpy().astype(np.uint64)


def _t(a):
    return torch.from_numpy(np.asarray(a, dtype=np.uint64).astype(np.int64))


class OracleOps:
    """Codes as int64 CPU tensors (b <= 31)."""

    def column_max(self, c0, c1):
        a = np.concatenate([c0.numpy().view(np.uint32), c1.numpy().view(np.uint32)])
        return int(a.max()) if a.size else 0

    def encode(self, c0, c1, b, wide):
        return _t((c0.numpy().view(np.uint32).astype(np.uint64) << np.uint64(b)) |
                  c1.numpy().view(np.uint32).astype(np.uint64))

    def partition(self, codes, b, key_col, nparts):
        c = _np(codes)
        key = (c >> np.uint64(b)) if key_col == 0 else (c & np.uint64((1 << b) - 1))
        own = owner(key, nparts)
        order = np.argsort(own, kind="stable")
        return _t(c[order]), [int(x) for x in np.bincount(own, minlength=nparts)]

    def sort_unique(self, codes, key_bits):
        return _t(P.sort_unique_codes(_np(codes)))

    def difference_merge(self, full, fresh):
        d, f = P.difference_merge_codes(_np(full), _np(fresh))
        return _t(d), _t(f)

    def join_reach(self, delta, inner, b):
        return _t(P.join_codes(_np(delta), _np(inner), b, 0, 3, 1))

    def empty_like(self, codes):
        return codes[:0]

    @staticmethod
    def size(codes):
        return int(codes.numel())


def decode(codes, b):
    c = np.asarray(codes, dtype=np.uint64)
    return (c >> np.uint64(b)).astype(np.uint32), (c & np.uint64((1 << b) - 1)).astype(np.uint32)
