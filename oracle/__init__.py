"""CPU oracle for batched MD5 / SHA-1 / SM3 -- TEST INFRASTRUCTURE ONLY.

A plain C implementation of RFC 1321, FIPS 180-4 and GB/T 32905-2016, one
message at a time and one padded byte at a time, reached through ctypes.  Only
the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never does, and the
two share no code.

Pins (tests/test_oracle.py): Python ``hashlib`` (OpenSSL's MD5, SHA-1, SM3) on
random and boundary-length inputs, a 50-digit evaluation of the MD5 sine
table, integer square roots for the SHA-1 constants, and the paper's data
totals (Sec. V-A.2) for the digest sizes.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MD5, SHA1, SM3 = 0, 1, 2
SLOT_BYTES = 32
_DIGEST_SIZE = {MD5: 16, SHA1: 20, SM3: 32}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_digest_size.restype = ctypes.c_size_t
        lib.oracle_digest_size.argtypes = [ctypes.c_int]
        lib.oracle_digest.restype = ctypes.c_int
        lib.oracle_digest.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        lib.oracle_md5_sine_table.restype = None
        lib.oracle_md5_sine_table.argtypes = [ctypes.c_void_p]
        lib.oracle_sha1_K.restype = ctypes.c_uint32
        lib.oracle_sha1_K.argtypes = [ctypes.c_uint]
        lib.oracle_hash_batch.restype = ctypes.c_int
        lib.oracle_hash_batch.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
            ctypes.c_int]
        _lib = lib
    return _lib


def digest_size(alg: int) -> int:
    return int(_load().oracle_digest_size(int(alg)))


def digest(alg: int, msg: bytes) -> bytes:
    """Digest of one message (RFC 1321 / FIPS 180-4 / GB/T 32905)."""
    lib = _load()
    size = lib.oracle_digest_size(int(alg))
    if size == 0:
        raise ValueError("unknown algorithm code %r" % (alg,))
    buf = ctypes.create_string_buffer(bytes(msg), max(len(msg), 1))
    out = ctypes.create_string_buffer(size)
    rc = lib.oracle_digest(int(alg), buf, len(msg), out)
    if rc != 0:
        raise RuntimeError("oracle_digest failed: %d" % rc)
    return out.raw


def md5_sine_table() -> list[int]:
    """T[1..64] of RFC 1321 Sec. 3.4 as the oracle computes it."""
    arr = np.zeros(64, dtype=np.uint32)
    _load().oracle_md5_sine_table(arr.ctypes.data)
    return [int(x) for x in arr]


def sha1_K(t: int) -> int:
    """K_t of FIPS 180-4 Sec. 4.2.1 as the oracle uses it."""
    return int(_load().oracle_sha1_K(int(t)))


def hash_batch(alg, packed: np.ndarray, offsets: np.ndarray, lengths: np.ndarray,
               algs: np.ndarray | None = None, threads: int = 1) -> np.ndarray:
    """Digest every message of a packed batch; returns an (n, 32) uint8 array.

    ``alg`` is one algorithm code for the whole batch, or ignored when
    ``algs`` (uint8 per message) is given.  Slot i holds the digest of
    ``packed[offsets[i]:offsets[i]+lengths[i]]`` followed by zero bytes.
    """
    lib = _load()
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    n = int(offsets.shape[0])
    if lengths.shape[0] != n:
        raise ValueError("offsets and lengths differ in length")
    algs_ptr = None
    if algs is not None:
        algs = np.ascontiguousarray(algs, dtype=np.uint8)
        if algs.shape[0] != n:
            raise ValueError("algs must have one entry per message")
        algs_ptr = algs.ctypes.data
    out = np.zeros((n, SLOT_BYTES), dtype=np.uint8)
    rc = lib.oracle_hash_batch(
        -1 if alg is None else int(alg), algs_ptr,
        packed.ctypes.data if packed.size else None, int(packed.size),
        offsets.ctypes.data if n else None, lengths.ctypes.data if n else None,
        n, out.ctypes.data if n else None, int(threads))
    if rc == -1:
        raise ValueError("unknown algorithm code in batch")
    if rc == -2:
        raise ValueError("message outside the packed buffer")
    if rc != 0:
        raise RuntimeError("oracle_hash_batch failed: %d" % rc)
    return out


def host_threads() -> int:
    return len(os.sched_getaffinity(0))
