"""Splitting one batch across GPUs by estimated work.

Messages are independent, so a batch shards with no exchange: rank r hashes a
contiguous range of message indices and writes its own range of digest slots.
Ranges are balanced by estimated work rather than by count: a message costs
its padded block count (message + 0x80 + 8 length bytes, rounded up to 64;
RFC 1321 Sec. 3.1-3.2, FIPS 180-4 Sec. 5.1.1, GB/T 32905 Sec. 5.2) times the
per-block cost of its algorithm, and the boundaries fall where the prefix sum
of those costs crosses r / parts of the total.  This is the device-level
counterpart of the paper's workload split between processors (Sec. IV-B),
with the measured per-block cost in place of its hardware ratio.
"""
from __future__ import annotations

import numpy as np

# 32-bit operations per 64-byte block (MD5, SHA-1, SM3), counted from the
# definitions as the kernels execute them.
OPS_PER_BLOCK = np.array([324, 613, 1412], dtype=np.int64)


def padded_blocks(lengths) -> np.ndarray:
    return (np.asarray(lengths, dtype=np.int64) + 72) // 64


def message_costs(lengths, algs=None, alg: int | None = None) -> np.ndarray:
    """Estimated work of each message: padded blocks x ops per block of its
    algorithm (per-message codes `algs`, or one `alg` for all)."""
    nb = padded_blocks(lengths)
    if algs is None:
        if alg is None:
            raise ValueError("give algs or alg")
        return nb * OPS_PER_BLOCK[int(alg)]
    codes = np.asarray(algs, dtype=np.int64)
    valid = codes <= 2
    cost = np.zeros(nb.shape, dtype=np.int64)
    cost[valid] = nb[valid] * OPS_PER_BLOCK[codes[valid]]
    return cost


def partition(costs, parts: int) -> list[tuple[int, int]]:
    """Contiguous index ranges [start, end), one per part, that split the
    total cost as evenly as contiguous ranges allow (boundaries where the
    prefix sum crosses k/parts of the total)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    costs = np.asarray(costs, dtype=np.int64)
    n = costs.shape[0]
    if n == 0:
        return [(0, 0)] * parts
    prefix = np.cumsum(costs)
    total = int(prefix[-1])
    bounds = [0]
    for k in range(1, parts):
        target = total * k / parts
        # first index whose inclusive prefix reaches the target, then pick
        # the closer of the two neighbouring cut points
        i = int(np.searchsorted(prefix, target, side="left"))
        cut = i + 1 if i < n else n
        if i < n and i > 0 and abs(prefix[i - 1] - target) <= abs(prefix[i] - target):
            cut = i
        bounds.append(max(bounds[-1], min(cut, n)))
    bounds.append(n)
    return [(bounds[k], bounds[k + 1]) for k in range(parts)]


def rank_range(lengths, algs=None, alg: int | None = None, rank: int = 0,
               world: int = 1) -> tuple[int, int]:
    """The message range rank `rank` of `world` hashes."""
    return partition(message_costs(lengths, algs, alg), world)[rank]
