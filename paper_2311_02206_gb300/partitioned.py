"""Hash-partitioned semi-naive REACH over several GPUs (one process per GPU).

The paper evaluates on one GPU and names a distributed, MPI-style semi-naive
evaluation as future work (its conclusion, after the distributed relational
algebra work it cites).  Restated for GPUs that exchange over NCCL:

* REACH(f, t) is partitioned by its first column: the tuple belongs to the
  GPU owner(f) = fmix32(f) mod P.  Delta tuples (m, t), read as the outer
  relation of Reach(f, t) <- Edge(f, m), Reach(m, t), therefore sit on the
  owner of their join column m.
* Edge is partitioned by its join column too: the inner tuples (m, f) sit on
  owner(m), so every GPU joins its own delta with its own part of Edge
  (Algorithm 3, no remote reads).
* One all-to-all per iteration sends each new tuple (f, t) to owner(f); the
  owner sorts and deduplicates what it received, takes the set difference
  against its part of full and merges (Section 5.1's populate-delta and merge).
* The sum of |delta_k| over the GPUs (an all-reduce) is the termination test
  and the iteration's delta count, so the delta counts equal those of the
  one-GPU evaluation and the union of the parts is the one-GPU relation.

Every data-parallel step is a call into libhisa.so (``CudaPartOps``): encode,
hash partition, join, sort + unique, difference + merge.  The exchange is
``torch.distributed`` (``TorchExchange``; all_to_all_single and all_reduce),
or, for several partitions held by one process, plain slicing and
concatenation (``LocalExchange``).  The iteration logic (``reach_partitioned``)
only calls these two interfaces, so it can be exercised on CPU ranks with
another implementation of the per-partition steps.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


class CudaPartOps:
    """The per-partition steps, each one libhisa.so call on torch CUDA tensors
    (codes: int32 tensors holding uint32 bit patterns, or int64)."""

    def __init__(self, stream=None):
        from . import hisa
        self.h = hisa
        self.stream = stream

    def column_max(self, c0, c1) -> int:
        return self.h.column_max(c0, c1, self.stream)

    def encode(self, c0, c1, b: int, wide: bool):
        return self.h.encode_codes(c0, c1, b, wide, self.stream)

    def partition(self, codes, b: int, key_col: int, nparts: int):
        return self.h.partition_codes(codes, b, key_col, nparts, self.stream)

    def sort_unique(self, codes, key_bits: int):
        return self.h.sort_unique_codes(codes, key_bits, self.stream)

    def difference_merge(self, full, fresh):
        return self.h.difference_merge(full, fresh, True, self.stream)

    def join_reach(self, delta, inner, b: int):
        """delta (m, t) joined on m with inner (m, f): results (f, t) (Algorithm 3)."""
        return self.h.join_codes(delta, inner, b, 0, 3, 1, 0, self.stream)

    def empty_like(self, codes):
        return codes[:0]

    @staticmethod
    def size(codes) -> int:
        return int(codes.numel())


class TorchExchange:
    """One partition per rank of a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.nparts = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.local = [self.rank]

    def _dev(self, like):
        return like.device

    def all_to_all(self, sends: List[Tuple[object, List[int]]]):
        import torch
        (send, counts), = sends
        dev = self._dev(send)
        scounts = torch.tensor(counts, dtype=torch.int64, device=dev)
        rcounts = torch.empty(self.nparts, dtype=torch.int64, device=dev)
        self.dist.all_to_all_single(rcounts, scounts, group=self.group)
        rc = [int(x) for x in rcounts.cpu().tolist()]
        recv = torch.empty(sum(rc), dtype=send.dtype, device=dev)
        self.dist.all_to_all_single(recv, send[:sum(counts)], rc, list(counts), group=self.group)
        return [recv]

    def _reduce(self, x: int, op, like):
        import torch
        t = torch.tensor([x], dtype=torch.int64, device=self._dev(like))
        self.dist.all_reduce(t, op=op, group=self.group)
        return int(t.item())

    def allreduce_sum(self, x: int, like) -> int:
        return self._reduce(x, self.dist.ReduceOp.SUM, like)

    def allreduce_max(self, x: int, like) -> int:
        return self._reduce(x, self.dist.ReduceOp.MAX, like)


class LocalExchange:
    """All `nparts` partitions held by this process (one GPU or a test): the
    all-to-all is slicing and concatenation, the reductions are sums."""

    def __init__(self, nparts: int):
        self.nparts = nparts
        self.rank = 0
        self.local = list(range(nparts))

    def all_to_all(self, sends):
        import torch
        recv = []
        for q in range(self.nparts):
            pieces = []
            for send, counts in sends:
                lo = sum(counts[:q])
                pieces.append(send[lo:lo + counts[q]])
            recv.append(torch.cat(pieces) if pieces else sends[0][0][:0])
        return recv

    def allreduce_sum(self, x: int, like) -> int:
        return x

    def allreduce_max(self, x: int, like) -> int:
        return x


def reach_partitioned(edges: Sequence[Tuple[object, object]], ops, ex, max_iters: int = 1 << 20):
    """REACH over the partitions of `ex`.

    edges: one (c0, c1) column pair per partition this process holds (ex.local):
    its share of Edge(f, t), any split of the edge list over the partitions.
    Returns (full, b, delta_counts): per local partition its tuples of Reach
    as sorted codes (f << b) | t -- exactly those with owner(f) equal to the
    partition -- the domain bits, and |delta_1| .. |delta_K| over all partitions."""
    P = ex.nparts
    assert len(edges) == len(ex.local)
    like = edges[0][0]
    mx = max(ops.column_max(c0, c1) for c0, c1 in edges)
    mx = ex.allreduce_max(mx, like)
    b = max(1, int(mx).bit_length())
    wide = 2 * b > 32
    kbits = 2 * b

    def exchange(codes_list, key_col):
        return ex.all_to_all([ops.partition(c, b, key_col, P) for c in codes_list])

    # the join's inner relation: Edge as (m, f) on owner(m), sorted and deduplicated
    inner = [ops.sort_unique(r, kbits) for r in exchange([ops.encode(c1, c0, b, wide) for c0, c1 in edges], 0)]
    # iteration 1 (the non-recursive rule): delta_1 = Edge as (f, t) on owner(f)
    fresh = [ops.sort_unique(r, kbits) for r in exchange([ops.encode(c0, c1, b, wide) for c0, c1 in edges], 0)]
    full, delta = [], []
    for x in fresh:
        d, f = ops.difference_merge(ops.empty_like(x), x)
        delta.append(d)
        full.append(f)
    counts = []
    total = ex.allreduce_sum(sum(ops.size(d) for d in delta), like)
    it = 1
    while total > 0:
        counts.append(total)
        if it >= max_iters:
            raise RuntimeError("no fixpoint within max_iters iterations")
        it += 1
        # join each partition's delta (m, t) with its Edge part (m, f): (f, t)
        new = [ops.join_reach(d, i, b) for d, i in zip(delta, inner)]
        # to the owners of f; each owner: sort + unique, difference, merge
        fresh = [ops.sort_unique(r, kbits) for r in exchange(new, 0)]
        delta = []
        for p, x in enumerate(fresh):
            d, f = ops.difference_merge(full[p], x)
            delta.append(d)
            full[p] = f
        total = ex.allreduce_sum(sum(ops.size(d) for d in delta), like)
    return full, b, counts
