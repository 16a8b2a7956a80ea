"""The relay form of the fused kernel (few long messages, chains passed from
warp to warp between segments) against the oracle, bit-exact.

A batch of between 2 and 8 x 32 messages per SM sub-partition takes the
relay; these batches sit inside that window on a 148-SM device.  Lengths
straddle every segment boundary (a segment that is not the last is pure data;
the last holds the rest and the padding, one block more than a segment when
the data ends just short of a boundary).
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


def _relay_window(hb):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return 2 * sms * 32, 8 * 4 * sms * 32       # messages: [half, eight] chunks per sub-partition


def _lengths(seg_bytes, n, seed):
    # boundary lengths around 1..4 segments, then log-uniform up to 40 KiB
    base = []
    for k in range(1, 5):
        e = k * seg_bytes
        base += [e - 65, e - 64, e - 57, e - 56, e - 55, e - 9, e - 8, e - 1, e, e + 1, e + 55,
                 e + 56, e + 63, e + 64]
    base += [0, 1, 55, 56, 63, 64, 119, 120]
    rng = np.random.Generator(np.random.PCG64(seed))
    rest = workloads.ragged_lengths(rng, n - len(base), max_len=40 << 10)
    lens = np.concatenate([np.asarray(base, dtype=np.int64).clip(0), rest.astype(np.int64)])
    return rng.permutation(lens).astype(np.uint32)


def _oracle_records(oracle_mod, b):
    return [oracle_mod.hash_batch(alg, b.packed, b.offsets, b.lengths,
                                  threads=oracle_mod.host_threads()) for alg in ALGS]


def _assert_records(rec, want, where):
    for alg in ALGS:
        got = rec[:, 32 * alg:32 * alg + 32]
        if not np.array_equal(got, want[alg]):
            bad = np.nonzero((got != want[alg]).any(axis=1))[0]
            raise AssertionError("%s alg %d: %d of %d records differ, first at %s"
                                 % (where, alg, bad.size, len(got), bad[:8]))


def _kernel_names(fn):
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    return {e.name for e in prof.events()}


@pytest.mark.parametrize("seg_blocks", [32, 3, 1])
def test_relay_equals_oracle_and_grid_stride(hb, oracle_mod, seg_blocks):
    lo, hi = _relay_window(hb)
    n = lo + 77                                   # a ragged last chunk, inside the window
    assert n <= hi and hb.all_uses_relay(n)
    b = workloads.scattered(_lengths(seg_blocks * 64, n, seed=300 + seg_blocks), seed=7, overlap=True)
    packed, off, ln, _ = hb.to_device(b)
    want = _oracle_records(oracle_mod, b)
    hb.tune_relay(seg_blocks)
    try:
        rec = torch.full((b.n, 96), 0xA5, dtype=torch.uint8, device="cuda")
        names = _kernel_names(lambda: hb.hash_batch_all(packed, off, ln, out=rec))
        assert any("hb_relay_kernel" in k for k in names), sorted(names)
        assert hb.device_status() == 0
        _assert_records(rec.cpu().numpy(), want, "relay seg %d" % seg_blocks)
        # the grid-stride kernel gives the same records
        hb.tune_relay(0)
        rec2 = torch.zeros((b.n, 96), dtype=torch.uint8, device="cuda")
        names = _kernel_names(lambda: hb.hash_batch_all(packed, off, ln, out=rec2))
        assert not any("hb_relay_kernel" in k for k in names)
        assert torch.equal(rec, rec2)
    finally:
        hb.tune_relay(64)


def test_relay_at_the_window_edges_and_repeated(hb, oracle_mod):
    # the smallest and the largest batch the relay takes, equal lengths (the
    # long-message workload's shape), each hashed twice into a buffer that
    # still holds the first call's records (the blocks-done words are reset)
    lo, hi = _relay_window(hb)
    for n, length in ((lo, 4100), (hi, 300)):
        b = workloads.fixed(n, length, seed=n)
        packed, off, ln, _ = hb.to_device(b)
        want = _oracle_records(oracle_mod, b)
        rec = torch.empty((b.n, 96), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            hb.hash_batch_all(packed, off, ln, out=rec)
            torch.cuda.synchronize()
            assert hb.device_status() == 0
            _assert_records(rec.cpu().numpy(), want, "relay n %d" % n)


def test_relay_window(hb):
    lo, hi = _relay_window(hb)
    assert hb.all_uses_relay(lo) and hb.all_uses_relay(hi) and hb.all_uses_relay(65536)
    assert not hb.all_uses_relay(lo - 32) and not hb.all_uses_relay(hi + 1)
    assert not hb.all_uses_relay(1 << 22)         # the short-message step: grid-stride kernel
    hb.tune_relay(0)
    try:
        assert not hb.all_uses_relay(65536)
    finally:
        hb.tune_relay(64)


def test_relay_argument_checks(hb):
    from paper_2407_09333_b300.api import HashBatchError
    with pytest.raises(HashBatchError):
        hb.tune_relay(-1)
    with pytest.raises(HashBatchError):
        hb.tune_relay((1 << 20) + 1)
    hb.tune_relay(64)


def test_relay_wait_limit_reports_a_timeout(hb):
    # The relay's wait for a previous segment is bounded.  With a 1 ns limit
    # and more warps than chunks (the smallest relay batch, one-block
    # segments) some warp is bound to find its count not yet reached: the
    # wait gives up, the launch still ends, and the device status carries
    # HB_DEV_TIMEOUT (the digests are then not to be trusted).  Nothing here
    # faults: every address the kernel touches stays valid.
    lo, _ = _relay_window(hb)
    b = workloads.fixed(lo, 8192, seed=17)
    packed, off, ln, _ = hb.to_device(b)
    rec = torch.empty((b.n, 96), dtype=torch.uint8, device="cuda")
    assert hb.device_status() == 0
    hb.tune_relay(1)
    old = hb.set_wait_limit_ns(1)
    try:
        hb.hash_batch_all(packed, off, ln, out=rec)
        torch.cuda.synchronize()
    finally:
        hb.set_wait_limit_ns(old)
        hb.tune_relay(64)
    assert hb.device_status() & hb.DEV_TIMEOUT          # read and cleared
    assert hb.device_status() == 0
    hb.hash_batch_all(packed, off, ln, out=rec)         # and the next call is clean
    torch.cuda.synchronize()
    assert hb.device_status() == 0


@pytest.mark.parametrize("shape", [6, 11])
def test_relay_with_four_block_stages(hb, oracle_mod, shape):
    # the benchmark's relay shape (8 warps, 2 stages of 4 blocks, per-lane
    # copies) and its cooperative-copy twin, with 3-block segments: every
    # segment ends part-way through a stage
    lo, _ = _relay_window(hb)
    n = lo + 13
    b = workloads.scattered(_lengths(3 * 64, n, seed=500 + shape), seed=21, overlap=True)
    packed, off, ln, _ = hb.to_device(b)
    want = _oracle_records(oracle_mod, b)
    hb.tune_relay(3)
    try:
        rec = torch.full((b.n, 96), 0x3C, dtype=torch.uint8, device="cuda")
        names = _kernel_names(lambda: hb.hash_batch_all(packed, off, ln, out=rec, shape=shape))
        assert any("hb_relay_kernel" in k for k in names), sorted(names)
        assert hb.device_status() == 0
        _assert_records(rec.cpu().numpy(), want, "relay shape %d" % shape)
    finally:
        hb.tune_relay(64)


def test_relay_calls_on_two_streams_share_the_counter_in_order(hb, oracle_mod):
    # two relay batches issued back to back on two streams without a host
    # synchronisation: the per-device item counter is reset by each call's
    # setup, so the second call must wait for the first (the library orders
    # them with an event), and both must come out right
    lo, _ = _relay_window(hb)
    batches = [workloads.scattered(_lengths(64 * 64, lo + 5 + 7 * k, seed=600 + k), seed=30 + k,
                                   overlap=True) for k in range(2)]
    dev = [hb.to_device(b) for b in batches]
    want = [_oracle_records(oracle_mod, b) for b in batches]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    recs = [torch.empty((b.n, 96), dtype=torch.uint8, device="cuda") for b in batches]
    torch.cuda.synchronize()
    for (packed, off, ln, _), rec, st in zip(dev, recs, streams):
        with torch.cuda.stream(st):
            hb.hash_batch_all(packed, off, ln, out=rec, stream=st)
    torch.cuda.synchronize()
    assert hb.device_status() == 0
    for k, (rec, w) in enumerate(zip(recs, want)):
        _assert_records(rec.cpu().numpy(), w, "stream %d" % k)
