"""Seeded synthetic inputs for the batched-hash path.

This module only draws bytes, lengths, offsets and algorithm codes with numpy's
PCG64; it holds none of the hashing arithmetic (no padding, no block counts,
no digests), so both the CPU oracle and the CUDA library can be fed from it.

Shapes follow the paper's workload (Sec. V-A.2: a very large number of short
independent messages, each hashed into its own digest slot) and the five
configurations the library is measured on:

* ``fixed(n, L, seed)``      -- n messages of exactly L bytes, packed back to
  back (offsets L*i, so unaligned whenever L is not a multiple of 16).
* ``ragged(n, seed)``         -- lengths floor(exp(U(0, ln 65537))) - 1 in
  [0, 65536], 1% of the messages forced to a padding-boundary length,
  per-message algorithm uniform in {MD5, SHA-1, SM3}, packed back to back in
  a shuffled order.
* ``digits9(n, first)``       -- the paper's own message shape: 9-character
  decimal strings, consecutive values starting at ``first``.
* ``scattered(...)``          -- unaligned offsets with gaps and overlaps, for
  layout tests.
* ``serve_requests(...)``     -- Poisson arrivals of mixed requests.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BOUNDARY_LENGTHS = (0, 55, 56, 63, 64, 119, 120)


@dataclasses.dataclass
class Batch:
    packed: np.ndarray          # uint8, the packed message bytes
    offsets: np.ndarray         # uint64, start of message i in `packed`
    lengths: np.ndarray         # uint32, byte length of message i
    algs: np.ndarray | None = None  # uint8 per message (mixed batches only)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0])

    @property
    def total_bytes(self) -> int:
        return int(self.lengths.astype(np.uint64).sum())


def _random_bytes(rng: np.random.Generator, size: int) -> np.ndarray:
    """`size` uniform random bytes: the raw 64-bit PCG64 outputs, little-endian."""
    if size == 0:
        return np.zeros(0, dtype=np.uint8)
    words = rng.bit_generator.random_raw((size + 7) // 8)
    return words.view(np.uint8)[:size]


def fixed(n: int, length: int, seed: int) -> Batch:
    """n messages of `length` uniform random bytes packed back to back."""
    rng = np.random.Generator(np.random.PCG64(seed))
    packed = _random_bytes(rng, n * length)
    offsets = np.arange(n, dtype=np.uint64) * np.uint64(length)
    lengths = np.full(n, length, dtype=np.uint32)
    return Batch(packed, offsets, lengths)


def ragged_lengths(rng: np.random.Generator, n: int, max_len: int = 65536,
                   boundary_frac: float = 0.01) -> np.ndarray:
    """Log-uniform lengths in [0, max_len] with a share forced to boundaries."""
    u = rng.uniform(0.0, np.log(max_len + 1.0), size=n)
    lengths = np.floor(np.exp(u)).astype(np.int64) - 1
    lengths = np.clip(lengths, 0, max_len)
    k = int(round(boundary_frac * n))
    if k:
        idx = rng.choice(n, size=k, replace=False)
        lengths[idx] = rng.choice(np.asarray(BOUNDARY_LENGTHS, dtype=np.int64), size=k)
    return lengths.astype(np.uint32)


def ragged(n: int, seed: int, max_len: int = 65536, boundary_frac: float = 0.01) -> Batch:
    """Mixed-algorithm ragged batch, messages laid out in shuffled order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = ragged_lengths(rng, n, max_len, boundary_frac)
    algs = rng.integers(0, 3, size=n, dtype=np.uint8)
    order = rng.permutation(n)                    # position -> message id
    starts = np.zeros(n, dtype=np.uint64)
    laid = lengths[order].astype(np.uint64)
    if n:
        starts[1:] = np.cumsum(laid)[:-1]
    offsets = np.empty(n, dtype=np.uint64)
    offsets[order] = starts
    packed = _random_bytes(rng, int(laid.sum()))
    return Batch(packed, offsets, lengths, algs)


def digits9(n: int, first: int = 0) -> Batch:
    """9-character decimal strings first, first+1, ... (paper Sec. V-A.2)."""
    vals = (np.arange(n, dtype=np.int64) + first) % 1_000_000_000
    digits = np.empty((n, 9), dtype=np.uint8)
    for k in range(8, -1, -1):
        digits[:, k] = (vals % 10).astype(np.uint8) + ord("0")
        vals //= 10
    packed = digits.reshape(-1).copy()
    offsets = np.arange(n, dtype=np.uint64) * np.uint64(9)
    lengths = np.full(n, 9, dtype=np.uint32)
    return Batch(packed, offsets, lengths)


def scattered(lengths, seed: int, overlap: bool = True, mixed: bool = False) -> Batch:
    """Messages at random unaligned offsets, with gaps and (optionally) overlaps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = np.asarray(lengths, dtype=np.uint32)
    n = int(lengths.shape[0])
    total = int(lengths.astype(np.uint64).sum())
    size = max(total + 4 * n + 64, 1)
    packed = _random_bytes(rng, size)
    if overlap:
        hi = np.maximum(size - lengths.astype(np.int64), 0)
        offsets = (rng.random(n) * (hi + 1)).astype(np.uint64)
    else:
        gaps = rng.integers(0, 4, size=n).astype(np.uint64)
        offsets = np.zeros(n, dtype=np.uint64)
        pos = np.uint64(0)
        for i in range(n):
            pos += gaps[i]
            offsets[i] = pos
            pos += np.uint64(lengths[i])
    algs = rng.integers(0, 3, size=n, dtype=np.uint8) if mixed else None
    return Batch(packed, offsets, lengths, algs)


@dataclasses.dataclass
class Request:
    arrival_s: float
    alg: int
    lengths: np.ndarray     # uint32 per message
    seed: int               # seed of this request's bytes

    @property
    def nbytes(self) -> int:
        return int(self.lengths.astype(np.uint64).sum())

    def payload(self) -> Batch:
        rng = np.random.Generator(np.random.PCG64(self.seed))
        n = int(self.lengths.shape[0])
        offsets = np.zeros(n, dtype=np.uint64)
        if n:
            offsets[1:] = np.cumsum(self.lengths.astype(np.uint64))[:-1]
        packed = _random_bytes(rng, self.nbytes)
        return Batch(packed, offsets, self.lengths.copy())


def serve_requests(count: int, rate_per_s: float, seed: int,
                   max_msgs: int = 4096, min_len: int = 16,
                   max_len: int = 1 << 20) -> list[Request]:
    """Poisson arrivals; each request has floor(exp(U(0, ln(max_msgs+1))))
    messages with log-uniform lengths in [min_len, max_len] and one algorithm."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        nmsg = int(np.floor(np.exp(rng.uniform(0.0, np.log(max_msgs + 1.0)))))
        nmsg = min(max(nmsg, 1), max_msgs)
        lens = np.floor(np.exp(rng.uniform(np.log(min_len), np.log(max_len + 1.0), size=nmsg)))
        lens = np.clip(lens, min_len, max_len).astype(np.uint32)
        alg = int(rng.integers(0, 3))
        out.append(Request(t, alg, lens, seed * 1_000_003 + k))
    return out
