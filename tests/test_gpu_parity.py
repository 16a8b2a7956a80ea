"""Parity of the CUDA path with the CPU oracle, slot by slot, bit-exact.

Digests are integer results with one correct value each, so the tolerance is
zero: every byte of every 32-byte slot (digest, then zero fill) must match.
Small cases are compared in full; the full-size batches (2^22 x 55 B,
65536 x 16 KiB, 2^20 ragged) are compared on seeded samples that the oracle
digests one message at a time, in the launch configuration the benchmark uses.
"""
import numpy as np
import pytest

from paper_2407_09333_b300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALGS = (0, 1, 2)


@pytest.fixture(scope="module")
def hb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09333_b300 import api, build
    build.build()
    api.lib()
    return api


def _oracle_slots(oracle_mod, batch, alg, idx=None):
    if idx is None:
        return oracle_mod.hash_batch(alg, batch.packed, batch.offsets, batch.lengths,
                                     algs=batch.algs, threads=oracle_mod.host_threads())
    algs = batch.algs[idx] if batch.algs is not None else None
    return oracle_mod.hash_batch(alg, batch.packed, batch.offsets[idx], batch.lengths[idx],
                                 algs=algs, threads=oracle_mod.host_threads())


def _gpu_slots(hb, batch, alg, shape=-1, mixed=False):
    packed, offsets, lengths, algs = hb.to_device(batch)
    if mixed:
        out = hb.hash_batch_mixed(algs, packed, offsets, lengths, shape=shape)
    else:
        out = hb.hash_batch(alg, packed, offsets, lengths, shape=shape)
    torch.cuda.synchronize()
    assert hb.device_status() == 0
    return out.cpu().numpy()


def _assert_slots_equal(got, want, where):
    if not np.array_equal(got, want):
        bad = np.nonzero((got != want).any(axis=1))[0]
        raise AssertionError("%s: %d of %d slots differ, first at %s" % (where, bad.size, len(want), bad[:8]))


@pytest.mark.parametrize("alg", ALGS)
def test_4096_by_64_bytes_seed0(hb, oracle_mod, alg):
    b = workloads.fixed(4096, 64, seed=0)
    _assert_slots_equal(_gpu_slots(hb, b, alg), _oracle_slots(oracle_mod, b, alg), "4096x64")


@pytest.mark.parametrize("alg", ALGS)
def test_every_length_0_to_300_packed_unaligned(hb, oracle_mod, alg):
    lens = list(range(0, 301)) + [511, 512, 513, 1000, 1023, 1024, 1025, 4095, 4096, 4097]
    b = workloads.scattered(lens, seed=11 + alg, overlap=False)
    _assert_slots_equal(_gpu_slots(hb, b, alg), _oracle_slots(oracle_mod, b, alg), "lengths")


@pytest.mark.parametrize("alg", ALGS)
def test_overlapping_unaligned_messages_all_shapes(hb, oracle_mod, alg):
    rng = np.random.default_rng(100 + alg)
    lens = rng.integers(0, 3000, size=1000)
    lens[:7] = workloads.BOUNDARY_LENGTHS
    b = workloads.scattered(lens, seed=21 + alg, overlap=True)
    want = _oracle_slots(oracle_mod, b, alg)
    for shape in range(len(hb.shapes())):
        _assert_slots_equal(_gpu_slots(hb, b, alg, shape=shape), want, "shape %d" % shape)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 65, 1000, 4097])
def test_ragged_warp_tails(hb, oracle_mod, n):
    b = workloads.fixed(n, 57, seed=n)
    for alg in ALGS:
        _assert_slots_equal(_gpu_slots(hb, b, alg), _oracle_slots(oracle_mod, b, alg), "n=%d" % n)


def test_long_messages(hb, oracle_mod):
    lens = [16384, 65536, 65537, 1 << 20, 100003, 0, 55, 120]
    b = workloads.scattered(lens, seed=5, overlap=False)
    for alg in ALGS:
        _assert_slots_equal(_gpu_slots(hb, b, alg), _oracle_slots(oracle_mod, b, alg), "long")


def test_nine_digit_messages(hb, oracle_mod):
    b = workloads.digits9(5000, first=999_995_000)   # wraps past 999999999
    for alg in ALGS:
        _assert_slots_equal(_gpu_slots(hb, b, alg), _oracle_slots(oracle_mod, b, alg), "digits9")


def test_empty_batch_is_noop(hb):
    packed = torch.zeros(16, dtype=torch.uint8, device="cuda")
    off = torch.zeros(0, dtype=torch.int64, device="cuda")
    ln = torch.zeros(0, dtype=torch.int32, device="cuda")
    out = hb.hash_batch(0, packed, off, ln)
    assert out.shape == (0, 32)
    out = hb.hash_batch_mixed(torch.zeros(0, dtype=torch.uint8, device="cuda"), packed, off, ln)
    assert out.shape == (0, 32)


def test_deterministic_and_same_alone_as_in_batch(hb, oracle_mod):
    b = workloads.scattered(np.arange(0, 700, 7), seed=3, overlap=True)
    g1 = _gpu_slots(hb, b, 2)
    g2 = _gpu_slots(hb, b, 2)
    assert np.array_equal(g1, g2)
    for i in (0, 17, 50, 99):
        one = workloads.Batch(b.packed, b.offsets[i:i + 1].copy(), b.lengths[i:i + 1].copy())
        assert np.array_equal(_gpu_slots(hb, one, 2)[0], g1[i])


# ---------------------------------------------------------------------------
# mixed / ragged path

def test_mixed_small_full_compare(hb, oracle_mod):
    b = workloads.ragged(20000, seed=7, max_len=8192)
    want = _oracle_slots(oracle_mod, b, None)
    _assert_slots_equal(_gpu_slots(hb, b, None, mixed=True), want, "mixed")


def test_mixed_all_shapes_and_invalid_codes(hb, oracle_mod):
    lens = np.random.default_rng(9).integers(0, 2000, size=3000)
    b = workloads.scattered(lens, seed=9, overlap=True, mixed=True)
    b.algs[::97] = 7          # unknown algorithm code: slot must stay zero
    ok = b.algs <= 2
    want = np.zeros((b.n, 32), dtype=np.uint8)
    idx = np.nonzero(ok)[0]
    want[idx] = _oracle_slots(oracle_mod, b, None, idx)
    for shape in range(len(hb.shapes())):
        _assert_slots_equal(_gpu_slots(hb, b, None, shape=shape, mixed=True), want, "shape %d" % shape)


@pytest.mark.parametrize("sub_log2,alg_major", [(0, 0), (2, 1), (3, 2), (4, 2), (5, 2), (6, 2), (6, 0)])
def test_mixed_every_bucketing_matches_oracle(hb, oracle_mod, sub_log2, alg_major):
    # bucket resolution and chunk order (including MD5's longest octave served
    # early from its own queue) change the schedule, never a digest
    lens = np.exp(np.random.default_rng(19).uniform(0, np.log(40000), size=6000)).astype(np.int64)
    b = workloads.scattered(lens, seed=19, overlap=True, mixed=True)
    want = _oracle_slots(oracle_mod, b, None)
    hb.tune_buckets(sub_log2, alg_major)
    try:
        _assert_slots_equal(_gpu_slots(hb, b, None, mixed=True), want,
                            "buckets %d,%d" % (sub_log2, alg_major))
        plan = hb.Plan(b.n)
        packed, off, ln, algs = hb.to_device(b)
        out = torch.zeros((b.n, 32), dtype=torch.uint8, device="cuda")
        plan.capture(algs, packed, off, ln, out)
        plan.replay(b.n)
        torch.cuda.synchronize()
        _assert_slots_equal(out.cpu().numpy(), want, "replayed %d,%d" % (sub_log2, alg_major))
        plan.close()
    finally:
        hb.tune_buckets(6, 2)


def test_mixed_matches_single_algorithm_path(hb):
    b = workloads.ragged(5000, seed=8, max_len=4096)
    mixed = _gpu_slots(hb, b, None, mixed=True)
    for alg in ALGS:
        sel = np.nonzero(b.algs == alg)[0]
        sub = workloads.Batch(b.packed, b.offsets[sel], b.lengths[sel])
        _assert_slots_equal(mixed[sel], _gpu_slots(hb, sub, alg), "alg %d" % alg)


# ---------------------------------------------------------------------------
# host-buffer path, bounds, failure detection

def test_standard_example_inputs(hb, oracle_mod):
    # ASCII inputs of the kind the standards' worked examples use, packed
    # back to back at odd offsets (expected slots from the oracle)
    alpha = "abcdefghijklmnopqrstuvwxyz"
    msgs = [b"", b"a", b"abc", b"message digest", alpha.encode(),
            (alpha.upper() + alpha + "0123456789").encode(),
            "".join(alpha[i:i + 4] for i in range(14)).encode(),
            "".join(alpha[i:i + 8] for i in range(14)).encode(),
            b"abcd" * 16, b"1234567890" * 8, b"a" * 1_000_000]
    packed = np.frombuffer(b"x" + b"".join(msgs) + b"x" * 16, dtype=np.uint8).copy()
    lengths = np.array([len(m) for m in msgs], dtype=np.uint32)
    offsets = (1 + np.concatenate([[0], np.cumsum(lengths)[:-1]])).astype(np.uint64)
    b = workloads.Batch(packed, offsets, lengths, None)
    for alg in ALGS:
        _assert_slots_equal(_gpu_slots(hb, b, alg), _oracle_slots(oracle_mod, b, alg), "examples")


@pytest.mark.parametrize("first,count", [(0, 1000), (77, 33), (123_456_703, 4_999),
                                         (999_999_000, 1000), (5, 1)])
def test_on_device_nine_digit_strings(hb, oracle_mod, first, count):
    # the paper's workload generated on the device, against the oracle over
    # the same strings laid out in memory
    b = workloads.digits9(count, first=first)
    for alg in ALGS:
        got = hb.hash_digits(alg, first, count).cpu().numpy()
        _assert_slots_equal(got, _oracle_slots(oracle_mod, b, alg), "digits %d+%d" % (first, count))


def _digit_strings(values):
    # the 9-character decimal strings of `values`, laid out back to back
    vals = np.asarray(values, dtype=np.int64) % 1_000_000_000
    digits = np.empty((vals.shape[0], 9), dtype=np.uint8)
    for k in range(8, -1, -1):
        digits[:, k] = (vals % 10).astype(np.uint8) + ord("0")
        vals = vals // 10
    n = digits.shape[0]
    return workloads.Batch(digits.reshape(-1).copy(), np.arange(n, dtype=np.uint64) * np.uint64(9),
                           np.full(n, 9, dtype=np.uint32), None)


def test_on_device_nine_digit_strings_several_passes(hb, oracle_mod):
    # more runs of ten strings than the grid holds at once (sms x 8 blocks x
    # 256 threads), starting off a multiple of ten: every thread and warp
    # makes a second pass over the grid stride, and MD5's warps reuse their
    # shared-memory staging.  Compared on every warp's first and last slot of
    # every pass, the batch ends and a seeded sample.
    first, count = 7, 4_000_003
    end = first + count
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    runs = (end + 9) // 10 - first // 10
    grid = max(1, min((runs + 255) // 256, sms * 8))
    assert runs > grid * 256, "the case must need more than one pass"
    warps = grid * 8
    qw = first // 10 + np.arange(0, runs, 32, dtype=np.int64)      # each warp-pass's first run
    heads = np.maximum(qw * 10, first)
    tails = np.minimum(qw * 10 + 319, end - 1)
    rng = np.random.default_rng(71)
    msgs = np.unique(np.concatenate([heads, tails, np.arange(first, first + 300),
                                     np.arange(end - 300, end), rng.integers(first, end, 20000)]))
    assert (qw.shape[0] + warps - 1) // warps >= 2
    sample = _digit_strings(msgs)
    k = torch.from_numpy(msgs - first).cuda()
    for alg in ALGS:
        out = hb.hash_digits(alg, first, count)
        got = out[k].cpu().numpy()
        _assert_slots_equal(got, _oracle_slots(oracle_mod, sample, alg), "digits passes alg %d" % alg)
        del out
    assert hb.device_status() == 0


def test_on_device_nine_digit_limits(hb):
    with pytest.raises(hb.HashBatchError) as e:
        hb.hash_digits(0, hb.DIGITS_COUNT - 5, 6)
    assert e.value.code == -3
    with pytest.raises(hb.HashBatchError) as e:
        hb.hash_digits(3, 0, 10)
    assert e.value.code == -1


@pytest.mark.parametrize("alg", [0, 1])
def test_bit_length_needs_the_high_word(hb, oracle_mod, alg):
    # 2^29 + 37 bytes: 8L no longer fits 32 bits, so the length block carries
    # a nonzero high word (little-endian for MD5, big-endian for SHA-1/SM3)
    L = (1 << 29) + 37
    b = workloads.fixed(1, L, seed=61)
    _assert_slots_equal(_gpu_slots(hb, b, alg), _oracle_slots(oracle_mod, b, alg), "2^29+37")


@pytest.mark.parametrize("shape", [0, 5, 10, 11, 14, 19])
def test_all_three_in_one_pass(hb, oracle_mod, shape):
    # every length 0..300 plus long ones, unaligned and overlapping: the
    # fused kernel's three slots equal the oracle's per-algorithm slots
    lens = list(range(0, 301)) + [511, 512, 513, 4095, 4096, 4097, 65537]
    b = workloads.scattered(lens, seed=41 + shape, overlap=True)
    packed, off, ln, _ = hb.to_device(b)
    rec = hb.hash_batch_all(packed, off, ln, shape=shape).cpu().numpy()
    assert rec.shape == (b.n, 96)
    for alg in ALGS:
        _assert_slots_equal(rec[:, 32 * alg:32 * alg + 32], _oracle_slots(oracle_mod, b, alg),
                            "all shape %d alg %d" % (shape, alg))


def test_all_three_host_path(hb, oracle_mod):
    b = workloads.fixed(20000, 55, seed=42)
    out = np.zeros((b.n, 96), dtype=np.uint8)
    hb.hash_batch_host(hb.ALL, b.packed, b.offsets, b.lengths, out)
    for alg in ALGS:
        _assert_slots_equal(out[:, 32 * alg:32 * alg + 32], _oracle_slots(oracle_mod, b, alg),
                            "all host alg %d" % alg)
    # through the device-memory windows as well
    old = hb.set_host_memory_limit(1 << 20)
    try:
        out2 = np.zeros_like(out)
        hb.hash_batch_host(hb.ALL, b.packed, b.offsets, b.lengths, out2)
    finally:
        hb.set_host_memory_limit(old)
    assert np.array_equal(out, out2)
    with pytest.raises(ValueError):
        hb.hash_batch_host(hb.ALL, b.packed, b.offsets, b.lengths, np.zeros((b.n, 32), np.uint8))


def test_host_path_plain_and_mixed(hb, oracle_mod):
    b = workloads.scattered(np.arange(0, 400), seed=4, overlap=True, mixed=True)
    out = np.zeros((b.n, 32), dtype=np.uint8)
    hb.hash_batch_host(None, b.packed, b.offsets, b.lengths, out, algs=b.algs)
    _assert_slots_equal(out, _oracle_slots(oracle_mod, b, None), "host mixed")
    plain = workloads.fixed(1000, 55, seed=1)
    out = np.zeros((plain.n, 32), dtype=np.uint8)
    hb.hash_batch_host(1, plain.packed, plain.offsets, plain.lengths, out)
    _assert_slots_equal(out, _oracle_slots(oracle_mod, plain, 1), "host plain")


@pytest.mark.parametrize("layout", ["packed", "shuffled"])
def test_host_path_pipelined_chunks(hb, oracle_mod, layout):
    # ~40 MB of packed bytes: the host path copies it in several chunks and
    # hashes each chunk's messages while later chunks are in flight.  In the
    # shuffled layout message ends are not in index order, so the chunk
    # assignment is wrong and the library must notice and hash again.
    rng = np.random.default_rng(21)
    lens = rng.integers(0, 9000, size=9000).astype(np.uint32)
    lens[:7] = workloads.BOUNDARY_LENGTHS
    b = workloads.scattered(lens, seed=22, overlap=False, mixed=True)
    offsets = b.offsets.copy()
    if layout == "shuffled":
        perm = rng.permutation(b.n)
        offsets, lens_p, algs_p = offsets[perm], b.lengths[perm], b.algs[perm]
        b = workloads.Batch(b.packed, offsets, lens_p, algs_p)
    for alg in (0, 2, None):
        out = np.zeros((b.n, 32), dtype=np.uint8)
        if alg is None:
            hb.hash_batch_host(None, b.packed, b.offsets, b.lengths, out, algs=b.algs)
        else:
            hb.hash_batch_host(alg, b.packed, b.offsets, b.lengths, out)
        sel = np.arange(0, b.n, 7)
        ref = b if alg is None else workloads.Batch(b.packed, b.offsets, b.lengths, None)
        want = _oracle_slots(oracle_mod, ref, alg, sel)
        _assert_slots_equal(out[sel], want, "host %s %s" % (layout, alg))


def test_host_path_streams_batches_over_the_memory_limit(hb, oracle_mod):
    # a 40 MB batch through two 2 MB device windows
    rng = np.random.default_rng(31)
    lens = rng.integers(0, 9000, size=9000).astype(np.uint32)
    lens[:7] = workloads.BOUNDARY_LENGTHS
    b = workloads.scattered(lens, seed=32, overlap=False, mixed=True)
    old = hb.set_host_memory_limit(4 << 20)
    try:
        sel = np.arange(0, b.n, 5)
        for alg in (1, None):
            out = np.zeros((b.n, 32), dtype=np.uint8)
            if alg is None:
                hb.hash_batch_host(None, b.packed, b.offsets, b.lengths, out, algs=b.algs)
                ref = b
            else:
                hb.hash_batch_host(alg, b.packed, b.offsets, b.lengths, out)
                ref = workloads.Batch(b.packed, b.offsets, b.lengths, None)
            _assert_slots_equal(out[sel], _oracle_slots(oracle_mod, ref, alg, sel), "windows %s" % alg)
        out = np.zeros((b.n, 32), dtype=np.uint8)
        # a layout that does not stream (ends out of order)
        perm = rng.permutation(b.n)
        with pytest.raises(hb.HashBatchError) as e:
            hb.hash_batch_host(2, b.packed, b.offsets[perm], b.lengths[perm], out)
        assert e.value.code == -10
        # a message outside the buffer
        offs = b.offsets.copy()
        offs[-1] = b.packed.size - 1
        with pytest.raises(hb.HashBatchError) as e:
            hb.hash_batch_host(2, b.packed, offs, b.lengths, out)
        assert e.value.code == -8
        # a message larger than a window
        big = workloads.fixed(3, 3 << 20, seed=33)
        with pytest.raises(hb.HashBatchError) as e:
            hb.hash_batch_host(0, big.packed, big.offsets, big.lengths, np.zeros((3, 32), np.uint8))
        assert e.value.code == -3
    finally:
        hb.set_host_memory_limit(old)
    # the library is still usable without the limit
    out = np.zeros((b.n, 32), dtype=np.uint8)
    hb.hash_batch_host(2, b.packed, b.offsets, b.lengths, out)
    ref = workloads.Batch(b.packed, b.offsets, b.lengths, None)
    _assert_slots_equal(out[:50], _oracle_slots(oracle_mod, ref, 2, np.arange(50)), "after")


@pytest.mark.parametrize("layout", ["packed", "shuffled"])
def test_host_path_packed_digests(hb, oracle_mod, layout):
    # Digests back to back on the host (16 / 20 / 32 bytes, 68 for all three):
    # the same bytes as the slots without their zero fill, over several copy
    # chunks, with message ends out of order (hashed again) and through the
    # device-memory windows.
    rng = np.random.default_rng(41)
    lens = rng.integers(0, 9000, size=9000).astype(np.uint32)
    lens[:7] = workloads.BOUNDARY_LENGTHS
    b = workloads.scattered(lens, seed=42, overlap=False, mixed=False)
    if layout == "shuffled":
        perm = rng.permutation(b.n)
        b = workloads.Batch(b.packed, b.offsets[perm], b.lengths[perm], None)
    sel = np.arange(0, b.n, 7)
    want = {alg: _oracle_slots(oracle_mod, b, alg, sel) for alg in ALGS}
    sizes = {0: 16, 1: 20, 2: 32}
    for alg in ALGS:
        out = np.zeros((b.n, sizes[alg]), dtype=np.uint8)
        hb.hash_batch_host(alg, b.packed, b.offsets, b.lengths, out, packed_digests=True)
        _assert_slots_equal(out[sel], want[alg][:, :sizes[alg]], "packed %s alg %d" % (layout, alg))
    out = np.zeros((b.n, hb.ALL_DIGEST_BYTES), dtype=np.uint8)
    hb.hash_batch_host(hb.ALL, b.packed, b.offsets, b.lengths, out, packed_digests=True)
    _assert_slots_equal(out[sel], np.concatenate([want[0][:, :16], want[1][:, :20], want[2]], axis=1),
                        "packed %s all" % layout)
    if layout == "packed":
        old = hb.set_host_memory_limit(4 << 20)
        try:
            out2 = np.zeros_like(out)
            hb.hash_batch_host(hb.ALL, b.packed, b.offsets, b.lengths, out2, packed_digests=True)
            out3 = np.zeros((b.n, 20), dtype=np.uint8)
            hb.hash_batch_host(1, b.packed, b.offsets, b.lengths, out3, packed_digests=True)
        finally:
            hb.set_host_memory_limit(old)
        assert np.array_equal(out, out2)
        _assert_slots_equal(out3[sel], want[1][:, :20], "packed windows sha1")
    with pytest.raises(ValueError):
        hb.hash_batch_host(0, b.packed, b.offsets, b.lengths, np.zeros((b.n, 8), np.uint8),
                           packed_digests=True)
    with pytest.raises(ValueError):
        hb.hash_batch_host(None, b.packed, b.offsets, b.lengths, np.zeros((b.n, 32), np.uint8),
                           algs=np.zeros(b.n, np.uint8), packed_digests=True)


def test_host_path_rejects_out_of_bounds(hb, oracle_mod):
    b = workloads.fixed(100, 40, seed=2)
    offs = b.offsets.copy()
    offs[50] = b.packed.size - 10          # runs 30 bytes past the end
    out = np.zeros((b.n, 32), dtype=np.uint8)
    with pytest.raises(hb.HashBatchError) as e:
        hb.hash_batch_host(0, b.packed, offs, b.lengths, out)
    assert e.value.code == -8
    # the library stays usable
    hb.hash_batch_host(0, b.packed, b.offsets, b.lengths, out)
    # a batch copied in several chunks whose last message runs past the end:
    # the call fails before hashing anything and the library stays usable
    big = workloads.fixed(4000, 10000, seed=3)       # 40 MB, five chunks
    offs = big.offsets.copy()
    offs[-1] = big.packed.size - 100
    out = np.zeros((big.n, 20), dtype=np.uint8)
    for packed_digests in (False, True):
        o = out if packed_digests else np.zeros((big.n, 32), np.uint8)
        with pytest.raises(hb.HashBatchError) as e:
            hb.hash_batch_host(1, big.packed, offs, big.lengths, o, packed_digests=packed_digests)
        assert e.value.code == -8
    hb.hash_batch_host(1, big.packed, big.offsets, big.lengths, out, packed_digests=True)
    ref = workloads.Batch(big.packed, big.offsets, big.lengths, None)
    sel = np.arange(0, big.n, 97)
    _assert_slots_equal(out[sel], _oracle_slots(oracle_mod, ref, 1, sel)[:, :20], "after bounds")


def test_check_bounds(hb):
    b = workloads.fixed(1000, 33, seed=6)
    _, off, ln, _ = hb.to_device(b)
    st = hb.check_bounds(off, ln, b.packed.size)
    assert int(st.item()) == 0
    st = hb.check_bounds(off, ln, b.packed.size - 1)
    assert int(st.item()) == hb.DEV_BOUNDS
    assert hb.device_status() & hb.DEV_BOUNDS
    assert hb.device_status() == 0        # cleared by the previous read


def test_bounded_wait_reports_timeout_and_context_survives(hb, oracle_mod):
    hb.device_status()
    hb.selftest_wait_timeout(20_000_000)   # 20 ms on a phase nothing completes
    assert hb.device_status() == hb.DEV_TIMEOUT
    b = workloads.fixed(64, 100, seed=12)
    _assert_slots_equal(_gpu_slots(hb, b, 0), _oracle_slots(oracle_mod, b, 0), "after timeout")


# ---------------------------------------------------------------------------
# full-size batches, sampled

def _sample(n, k, seed):
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([np.arange(min(n, 256)), np.arange(max(0, n - 256), n),
                                    rng.integers(0, n, size=k)]))
    return idx


def test_full_size_2pow22_by_55_sampled(hb, oracle_mod):
    b = workloads.fixed(1 << 22, 55, seed=1)
    packed, off, ln, _ = hb.to_device(b)
    idx = _sample(b.n, 20000, 1)
    for alg in ALGS:
        out = hb.hash_batch(alg, packed, off, ln)
        got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
        _assert_slots_equal(got, _oracle_slots(oracle_mod, b, alg, idx), "C2 alg %d" % alg)
    assert hb.device_status() == 0


def test_full_size_65536_by_16KiB_sampled(hb, oracle_mod):
    b = workloads.fixed(65536, 16384, seed=3)
    packed, off, ln, _ = hb.to_device(b)
    idx = _sample(b.n, 1500, 3)
    for alg in ALGS:
        out = hb.hash_batch(alg, packed, off, ln)
        got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
        _assert_slots_equal(got, _oracle_slots(oracle_mod, b, alg, idx), "C4 alg %d" % alg)


@pytest.mark.parametrize("n,length,seed,k", [(1 << 22, 55, 1, 20000), (65536, 16384, 3, 1500)])
def test_full_size_fused_sampled(hb, oracle_mod, tmp_path, n, length, seed, k):
    # the default benchmark step: the fused kernel in its autotuned shape
    from paper_2407_09333_b300 import autotune
    b = workloads.fixed(n, length, seed=seed)
    packed, off, ln, _ = hb.to_device(b)
    rec = torch.empty((b.n, 96), dtype=torch.uint8, device="cuda")
    autotune.tune(hb.ALL, packed, off, ln, rec, path=str(tmp_path / "tune.json"))
    hb.hash_batch_all(packed, off, ln, out=rec)
    idx = _sample(b.n, k, seed)
    got = rec[torch.from_numpy(idx).cuda()].cpu().numpy()
    for alg in ALGS:
        _assert_slots_equal(got[:, 32 * alg:32 * alg + 32], _oracle_slots(oracle_mod, b, alg, idx),
                            "fused %dx%d alg %d" % (n, length, alg))
    assert hb.device_status() == 0


@pytest.fixture(scope="module")
def c3(hb, oracle_mod):
    # the ragged benchmark batch: 2^20 messages, log-uniform lengths in
    # [0, 64 KiB], 1% at padding boundaries, algorithm per message (seed 2)
    b = workloads.ragged(1 << 20, seed=2)
    dev = hb.to_device(b)
    # the oracle's digests of a fixed sample: the first and last 256, 6000
    # seeded indices and every forced boundary-length message
    idx = _sample(b.n, 6000, 2)
    bl = np.nonzero(np.isin(b.lengths, workloads.BOUNDARY_LENGTHS))[0]
    idx = np.unique(np.concatenate([idx, bl]))
    want = _oracle_slots(oracle_mod, b, None, idx)
    yield b, dev, idx, want
    del dev
    torch.cuda.empty_cache()


def test_full_size_ragged_2pow20_sampled(hb, c3):
    b, (packed, off, ln, algs), idx, want = c3
    out = hb.hash_batch_mixed(algs, packed, off, ln)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    _assert_slots_equal(got, want, "C3")
    assert hb.device_status() == 0


def test_full_size_ragged_graph_replay_matches_oracle(hb, c3, tmp_path):
    # exactly the benchmark's ragged step: the autotuned shape, bucketing and
    # warps per SM, the launch sequence captured once as a graph, replayed with
    # the message count read on the device -- compared with the oracle, for
    # the whole batch and for prefixes (slots past the prefix stay untouched)
    from paper_2407_09333_b300 import autotune
    b, (packed, off, ln, algs), idx, want = c3
    out = torch.zeros((b.n, 32), dtype=torch.uint8, device="cuda")
    autotune.tune(None, packed, off, ln, out, algs=algs, path=str(tmp_path / "tune.json"))
    plan = hb.Plan(b.n)
    plan.capture(algs, packed, off, ln, out)
    try:
        for m in (b.n, 700_001, 65_536, 33, 1, b.n):
            out.zero_()
            plan.replay(m)
            torch.cuda.synchronize()
            sel = idx < m
            got = out[torch.from_numpy(idx[sel]).cuda()].cpu().numpy()
            _assert_slots_equal(got, want[sel], "C3 replay n=%d" % m)
            assert not bool(out[m:].any().item()), "slots past n=%d were written" % m
        assert hb.device_status() == 0
    finally:
        plan.close()
        hb.tune_set(hb.TUNE_MIXED, 19)
        hb.tune_buckets(6, 2)
        hb.tune_mixed_warps(8)


def test_autotuner_installs_a_valid_shape(hb, oracle_mod, tmp_path):
    from paper_2407_09333_b300 import autotune
    b = workloads.fixed(20000, 55, seed=13)
    packed, off, ln, _ = hb.to_device(b)
    out = torch.empty((b.n, 32), dtype=torch.uint8, device="cuda")
    path = str(tmp_path / "tune.json")
    r = autotune.tune(2, packed, off, ln, out, path=path)
    assert not r["cached"] and 0 <= r["shape"] < len(hb.shapes())
    assert hb.tune_get(2) == r["shape"]
    r2 = autotune.tune(2, packed, off, ln, out, path=path)
    assert r2["cached"] and r2["shape"] == r["shape"]
    got = hb.hash_batch(2, packed, off, ln).cpu().numpy()
    _assert_slots_equal(got, _oracle_slots(oracle_mod, b, 2), "tuned")
    hb.tune_set(2, 0)


def test_int_peak_microbenchmark_runs(hb):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for op in range(19):
        cyc = hb.int_peak(op, sms, 128, 10)
        torch.cuda.synchronize()
        assert int(cyc.min().item()) > 0


# ---------------------------------------------------------------------------
# plans: private scratch, concurrent streams, captured graphs

def test_plan_run_matches_mixed_path(hb):
    b = workloads.ragged(9000, seed=41, max_len=5000)
    packed, off, ln, algs = hb.to_device(b)
    want = hb.hash_batch_mixed(algs, packed, off, ln).cpu().numpy()
    plan = hb.Plan(b.n)
    out = torch.zeros((b.n, 32), dtype=torch.uint8, device="cuda")
    plan.run(algs, packed, off, ln, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    with pytest.raises(hb.HashBatchError):
        plan.run(algs, packed, off, ln, out, n=b.n + 1)
    plan.close()


def test_two_plans_on_two_streams(hb, oracle_mod):
    b1 = workloads.ragged(6000, seed=42, max_len=9000)
    b2 = workloads.ragged(4000, seed=43, max_len=3000)
    d1, d2 = hb.to_device(b1), hb.to_device(b2)
    p1, p2 = hb.Plan(b1.n), hb.Plan(b2.n)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    o1 = torch.zeros((b1.n, 32), dtype=torch.uint8, device="cuda")
    o2 = torch.zeros((b2.n, 32), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):
        p1.run(d1[3], d1[0], d1[1], d1[2], o1, stream=s1)
        p2.run(d2[3], d2[0], d2[1], d2[2], o2, stream=s2)
    torch.cuda.synchronize()
    _assert_slots_equal(o1.cpu().numpy(), _oracle_slots(oracle_mod, b1, None), "plan 1")
    _assert_slots_equal(o2.cpu().numpy(), _oracle_slots(oracle_mod, b2, None), "plan 2")
    p1.close()
    p2.close()


def test_captured_graph_replays_for_any_batch_size(hb):
    b = workloads.ragged(12000, seed=44, max_len=6000)
    packed, off, ln, algs = hb.to_device(b)
    plan = hb.Plan(b.n)
    out = torch.zeros((b.n, 32), dtype=torch.uint8, device="cuda")
    plan.capture(algs, packed, off, ln, out)
    for n in (b.n, 1, 33, 5000, b.n):
        out.zero_()
        plan.replay(n)
        torch.cuda.synchronize()
        want = hb.hash_batch_mixed(algs[:n].contiguous(), packed, off[:n].contiguous(),
                                   ln[:n].contiguous()).cpu().numpy()
        got = out.cpu().numpy()
        assert np.array_equal(got[:n], want), n
        assert not got[n:].any()
    with pytest.raises(hb.HashBatchError):
        plan.replay(b.n + 1)
    plan.close()
