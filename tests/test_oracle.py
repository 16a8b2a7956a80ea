"""Pins for the CPU oracle: checks against things other than the oracle itself.

* Python ``hashlib`` (OpenSSL's independent MD5 / SHA-1 / SM3) on every
  length 0..300, the padding boundaries, the paper's 9-digit messages and long
  inputs up to 1 MiB.
* The MD5 sine table against a 50-digit evaluation of floor(2^32 |sin i|)
  (RFC 1321 Sec. 3.4).
* The SHA-1 constants against integer square roots (FIPS 180-4 Sec. 4.2.1).
* The digest sizes against the paper's data totals (Sec. V-A.2).
* Batch layout invariants: batch slot == single-message digest, zero fill,
  overlapping / unaligned messages, error codes.
* Mutation check: a copy of the oracle with one planted mistake must fail at
  least one pin, for each of several plausible mistakes.
"""
import hashlib
import math
import os
import shutil
import subprocess
import ctypes

import numpy as np
import pytest

from paper_2407_09333_b300 import workloads

NAMES = {0: "md5", 1: "sha1", 2: "sm3"}
BOUNDARY = [0, 1, 3, 4, 9, 15, 16, 17, 55, 56, 57, 63, 64, 65, 119, 120, 121, 127, 128, 183, 184]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(seed, n):
    return np.random.default_rng(seed).integers(0, 256, n, dtype=np.uint8).tobytes()


@pytest.mark.parametrize("alg", [0, 1, 2])
def test_every_short_length_matches_hashlib(oracle_mod, alg):
    for L in range(0, 301):
        m = _rand(1000 * alg + L, L)
        assert oracle_mod.digest(alg, m) == hashlib.new(NAMES[alg], m).digest(), L


@pytest.mark.parametrize("alg", [0, 1, 2])
def test_boundary_and_long_lengths_match_hashlib(oracle_mod, alg):
    for L in BOUNDARY + [16384, 65536, 1 << 20]:
        m = _rand(7 + L, L)
        assert oracle_mod.digest(alg, m) == hashlib.new(NAMES[alg], m).digest(), L


@pytest.mark.parametrize("alg", [0, 1, 2])
def test_constant_bytes_match_hashlib(oracle_mod, alg):
    # all-zero and all-0xff messages stress the Boolean functions differently
    for L in (0, 55, 56, 64, 1000):
        for b in (0x00, 0xFF, 0x80):
            m = bytes([b]) * L
            assert oracle_mod.digest(alg, m) == hashlib.new(NAMES[alg], m).digest()


@pytest.mark.parametrize("alg", [0, 1, 2])
def test_standard_example_inputs_match_hashlib(oracle_mod, alg):
    # the kinds of input the standards' worked examples use: short ASCII
    # strings, the 56- and 112-byte alphabet runs that end exactly where
    # padding needs a second block, a 64-byte repeated pattern and a million
    # repeated bytes; expected digests come from hashlib, not from a table
    alpha = "abcdefghijklmnopqrstuvwxyz"
    msgs = [b"", b"a", b"abc", b"message digest", alpha.encode(),
            (alpha.upper() + alpha + "0123456789").encode(),
            "".join(alpha[i:i + 4] for i in range(14)).encode(),
            "".join(alpha[i:i + 8] for i in range(14)).encode(),
            b"abcd" * 16, b"1234567890" * 8, b"a" * 1_000_000]
    assert len(msgs[6]) == 56 and len(msgs[7]) == 112
    for m in msgs:
        assert oracle_mod.digest(alg, m) == hashlib.new(NAMES[alg], m).digest(), m[:16]


@pytest.mark.parametrize("alg", [0, 1, 2])
def test_paper_nine_digit_messages_match_hashlib(oracle_mod, alg):
    # the paper's message shape (Sec. V-A.2): 9 characters over {0-9}
    b = workloads.digits9(200, first=123_456_700)
    out = oracle_mod.hash_batch(alg, b.packed, b.offsets, b.lengths)
    d = oracle_mod.digest_size(alg)
    for i in range(b.n):
        m = b.packed[9 * i: 9 * i + 9].tobytes()
        assert m.isdigit() and len(m) == 9
        assert out[i, :d].tobytes() == hashlib.new(NAMES[alg], m).digest()


def test_md5_sine_table_against_50_digit_evaluation(oracle_mod):
    import mpmath
    mpmath.mp.dps = 50
    table = oracle_mod.md5_sine_table()
    for i in range(1, 65):
        exact = int(mpmath.floor(mpmath.mpf(2) ** 32 * abs(mpmath.sin(i))))
        assert table[i - 1] == exact, i


def test_sha1_constants_are_scaled_square_roots(oracle_mod):
    # K = floor(2^30 * sqrt(r)) = isqrt(r * 2^60) for r = 2, 3, 5, 10
    for t_range, r in ((range(0, 20), 2), (range(20, 40), 3), (range(40, 60), 5), (range(60, 80), 10)):
        want = math.isqrt(r << 60)
        for t in t_range:
            assert oracle_mod.sha1_K(t) == want, t


def test_digest_sizes_match_paper_data_totals(oracle_mod):
    rows = []
    with open(os.path.join(GOLDEN, "paper_data_totals.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                name, code, total = line.split()
                rows.append((name, int(code), float(total)))
    assert len(rows) == 3
    for name, code, total in rows:
        d = oracle_mod.digest_size(code)
        assert len(oracle_mod.digest(code, b"123456789")) == d
        assert round((9 + d) * 10**9 / 2**30, 2) == total, name


def test_batch_slots_equal_single_digests_with_overlaps(oracle_mod):
    lens = [0, 1, 55, 56, 63, 64, 65, 119, 120, 300, 1000, 4097] * 3
    b = workloads.scattered(lens, seed=5, overlap=True, mixed=True)
    out = oracle_mod.hash_batch(None, b.packed, b.offsets, b.lengths, algs=b.algs, threads=3)
    for i in range(b.n):
        alg = int(b.algs[i])
        m = b.packed[int(b.offsets[i]): int(b.offsets[i]) + int(b.lengths[i])].tobytes()
        d = oracle_mod.digest_size(alg)
        assert out[i, :d].tobytes() == hashlib.new(NAMES[alg], m).digest()
        assert not out[i, d:].any()


def test_batch_thread_count_does_not_change_result(oracle_mod):
    b = workloads.fixed(257, 70, seed=3)
    one = oracle_mod.hash_batch(2, b.packed, b.offsets, b.lengths, threads=1)
    many = oracle_mod.hash_batch(2, b.packed, b.offsets, b.lengths, threads=7)
    assert np.array_equal(one, many)


def test_batch_errors(oracle_mod):
    b = workloads.fixed(4, 10, seed=1)
    with pytest.raises(ValueError):
        oracle_mod.hash_batch(3, b.packed, b.offsets, b.lengths)
    bad = b.offsets.copy()
    bad[2] = 35  # 35 + 10 > 40
    with pytest.raises(ValueError):
        oracle_mod.hash_batch(0, b.packed, bad, b.lengths)
    empty = oracle_mod.hash_batch(0, b.packed, b.offsets[:0], b.lengths[:0])
    assert empty.shape == (0, 32)


# ---------------------------------------------------------------------------
# Planted mistakes: each mutant is a copy of the oracle with one plausible
# error; the hashlib pins above must catch every one of them.

MUTANTS = [
    ("padding.c", "8u * (7u - k) : 8u * k", "8u * k : 8u * (7u - k)"),   # length byte order
    ("padding.c", "return 0x80;", "return 0x01;"),                      # pad marker
    ("padding.c", "(len + 1 + 8 + 63) / 64", "(len + 8 + 63) / 64"),    # block count
    ("md5.c", "{7, 12, 17, 22}", "{7, 12, 17, 21}"),                    # one rotation
    ("md5.c", "(1u + 5u * j) % 16u", "(1u + 3u * j) % 16u"),            # word order
    ("md5.c", "(y & ~z)", "(~y & z)"),                                 # G function
    ("sha1.c", "oracle_rotl32(b, 30)", "oracle_rotl32(b, 29)"),
    ("sha1.c", "W[t - 14] ^ W[t - 16], 1)", "W[t - 14] ^ W[t - 16], 0)"),  # schedule rotate
    ("sha1.c", "if (t < 60) return sha1_Maj", "if (t < 59) return sha1_Maj"),
    ("sm3.c", "^ W[j - 6]", "^ W[j - 5]"),
    ("sm3.c", "Wp[j] = W[j] ^ W[j + 4]", "Wp[j] = W[j] ^ W[j + 3]"),
    ("sm3.c", "if (j < 16) return X ^ Y ^ Z;\n    return (X & Y) | (~X & Z);",
     "if (j < 15) return X ^ Y ^ Z;\n    return (X & Y) | (~X & Z);"),
    ("sm3.c", "V[7] ^= H;", "V[7] += H;"),
]


def _build_mutant(tmpdir, fname, old, new):
    src = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle")
    for f in os.listdir(src):
        if f.endswith((".c", ".h")):
            shutil.copy(os.path.join(src, f), tmpdir)
    path = os.path.join(tmpdir, fname)
    text = open(path).read()
    assert text.count(old) == 1, (fname, old)
    open(path, "w").write(text.replace(old, new))
    lib = os.path.join(tmpdir, "libmutant.so")
    srcs = [os.path.join(tmpdir, s) for s in ("padding.c", "md5.c", "sha1.c", "sm3.c", "batch.c")]
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-D_GNU_SOURCE", "-o", lib]
                   + srcs + ["-lm", "-lpthread"], check=True)
    return ctypes.CDLL(lib)


@pytest.mark.parametrize("mutant", range(len(MUTANTS)))
def test_planted_mistake_is_caught_by_pins(tmp_path, mutant):
    fname, old, new = MUTANTS[mutant]
    lib = _build_mutant(str(tmp_path), fname, old, new)
    lib.oracle_digest.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    caught = False
    for alg in (0, 1, 2):
        for L in BOUNDARY + [200]:
            m = _rand(L, L)
            buf = ctypes.create_string_buffer(m, max(L, 1))
            out = ctypes.create_string_buffer(32)
            lib.oracle_digest(alg, buf, L, out)
            want = hashlib.new(NAMES[alg], m).digest()
            if out.raw[:len(want)] != want:
                caught = True
                break
        if caught:
            break
    assert caught, "planted mistake %r not caught" % (MUTANTS[mutant],)
