"""Splitting one graph's count over several GPUs (host side).

The top-level sub-branches of EBBkC are independent (paper Sec. 6.2 (7), the
edge-parallel scheme), so N ranks that each hold a replica of the prepared graph can
each run a part of the ticket order -- the edges sorted by |VSet| descending --
through kc_params.ticket_begin / ticket_end, and add their results.  The order of
edges with equal |VSet| is not fixed from one prepare to another, so every cut falls
on a boundary between |VSet| sizes: a shard is a range of sizes, and the ticket range
of that size range is the same on every replica.  Sizes are assigned greedily so that
each shard's estimated cost is close to 1/N of the total.

The results combine exactly: counts are 128-bit integers, exchanged as 32-bit limbs
in 64-bit words (no limb sum can overflow for fewer than 2^31 ranks) and carried on the
host; checksums add mod 2^64.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1


def size_cost(s: np.ndarray, k: int) -> np.ndarray:
    """Estimated work of a top-level sub-branch of s vertices at k: the number of
    frames grows like s^(k-2) for small k and is bounded by the depth for large k; an
    exponent capped at 4 follows the measured per-edge cycles well enough to balance."""
    p = float(min(max(k - 2, 1), 4))
    return np.power(np.maximum(s.astype(np.float64), 1.0), p)


def _buckets(vset_sizes, k: int, nparts: int):
    vs = np.asarray(vset_sizes, dtype=np.int64)
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    live = vs[vs >= k - 2]
    sizes, counts = np.unique(live, return_counts=True)
    sizes, counts = sizes[::-1], counts[::-1]                 # descending, as the tickets
    bounds = [0]
    if sizes.size:
        cum_cost = np.cumsum(size_cost(sizes, k) * counts)
        total = float(cum_cost[-1])
        for r in range(1, nparts):
            # the size bucket whose cumulative cost reaches r/N of the total ends shard r-1
            j = int(np.searchsorted(cum_cost, total * r / nparts, side="left")) + 1
            bounds.append(max(bounds[-1], min(j, sizes.size)))
    else:
        bounds += [0] * (nparts - 1)
    bounds.append(sizes.size)
    return sizes, counts, bounds


def partition_by_size(vset_sizes, k: int, nparts: int) -> list[tuple[int, int]]:
    """Ticket ranges [begin, end) of nparts shards of the |VSet|-descending ticket order,
    cut only between different sizes, balanced by size_cost.  Edges with |VSet| < k-2
    (no k-clique) belong to no shard; ranges may be empty."""
    sizes, counts, bounds = _buckets(vset_sizes, k, nparts)
    cum_cnt = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return [(int(cum_cnt[bounds[r]]), int(cum_cnt[bounds[r + 1]])) for r in range(nparts)]


def shard_sizes(vset_sizes, k: int, nparts: int, r: int) -> np.ndarray:
    """The |VSet| sizes whose edges form shard r (the same shards as partition_by_size)."""
    sizes, _, bounds = _buckets(vset_sizes, k, nparts)
    return sizes[bounds[r]: bounds[r + 1]]


def to_limbs(count: int, checksum: int) -> list[int]:
    """(u128 count, u64 checksum) as six 32-bit limbs (low first)."""
    if count < 0 or count >= 1 << 128:
        raise ValueError("count out of range")
    return [(count >> (32 * i)) & 0xFFFFFFFF for i in range(4)] + \
           [(checksum >> (32 * i)) & 0xFFFFFFFF for i in range(2)]


def from_limbs(limbs) -> tuple[int, int]:
    """Inverse of to_limbs for limb-wise sums of several ranks (carries included)."""
    limbs = [int(x) for x in limbs]
    count = sum(limbs[i] << (32 * i) for i in range(4))
    checksum = (limbs[4] + (limbs[5] << 32)) & MASK64
    if count >= 1 << 128:
        raise OverflowError("the combined count reached 2^128")
    return count, checksum


def allreduce_result(count: int, checksum: int, group=None) -> tuple[int, int]:
    """Sum (count, checksum) over the ranks of a torch.distributed group, exactly."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(to_limbs(count, checksum), dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return from_limbs(t.cpu().tolist())
