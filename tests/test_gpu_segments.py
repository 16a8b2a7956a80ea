"""Segmented hashing: a message hashed piece by piece over several calls.

Merkle-Damgard hashing only carries the chaining value from one block to the
next (RFC 1321 Sec. 3.4, FIPS 180-4 Sec. 6.1.2, GB/T 32905 Sec. 5.3), so a
message cut at any block boundary and fed in order gives the digest of the
whole message.  These tests cut seeded messages at random block boundaries,
hash the pieces over several calls (each call holding one piece of every
unfinished message, in a shuffled order, next to messages that are hashed
whole) and compare every final slot with the CPU oracle's digest of the
whole message, bit for bit.
"""
import numpy as np
import pytest

from paper_2407_09333_b300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09333_b300 import api, build
    build.build()
    api.lib()
    return api


def _cuts(rng, length, max_pieces):
    """Piece sizes of one message: multiples of 64 except the last."""
    k = int(rng.integers(1, max_pieces + 1))
    if k == 1 or length < 64:
        return [length]
    bounds = np.sort(rng.integers(0, length // 64 + 1, size=k - 1)) * 64
    sizes = np.diff(np.concatenate([[0], bounds, [length]])).astype(np.int64)
    return [int(x) for x in sizes]


def _rounds(batch, rng, max_pieces):
    pieces = [_cuts(rng, int(L), max_pieces) for L in batch.lengths]
    return pieces, max(len(p) for p in pieces)


def _run_segmented(hb, batch, pieces, nrounds, rng, call, indexed=False):
    """Feeds round r's piece of every unfinished message; returns the final
    slots in message order (host numpy)."""
    n = batch.n
    packed = torch.from_numpy(np.ascontiguousarray(batch.packed)).cuda()
    if packed.numel() == 0:
        packed = torch.zeros(16, dtype=torch.uint8, device="cuda")
    slots_all = torch.full((n, 32), 0x5A, dtype=torch.uint8, device="cuda")
    done = np.zeros(n, dtype=bool)
    prior = np.zeros(n, dtype=np.uint64)
    for r in range(nrounds):
        active = np.array([i for i in range(n) if len(pieces[i]) > r], dtype=np.int64)
        rng.shuffle(active)
        if active.size == 0:
            continue
        sizes = np.array([pieces[i][r] for i in active], dtype=np.uint64)
        more = np.array([len(pieces[i]) > r + 1 for i in active])
        offs = batch.offsets[active] + prior[active]
        idx = torch.from_numpy(active).cuda()
        algs = torch.from_numpy(batch.algs[active]).cuda()
        off_t = torch.from_numpy(offs.astype(np.uint64).view(np.int64)).cuda()
        len_t = torch.from_numpy(sizes.astype(np.uint32).view(np.int32)).cuda()
        seg_t = torch.from_numpy(hb.seg_words(prior[active], more)).cuda()
        if indexed:
            # each message keeps its slot; the call maps positions to slots
            call(algs, packed, off_t, len_t, seg_t, slots_all, idx.to(torch.int32))
        else:
            slots = slots_all[idx].contiguous()       # this call's slot order
            call(algs, packed, off_t, len_t, seg_t, slots, None)
            slots_all[idx] = slots
        prior[active] += sizes
        done[active[~more]] = True
    torch.cuda.synchronize()
    assert done.all()
    assert hb.device_status() == 0
    return slots_all.cpu().numpy()


def _mixed_batch(n, seed, max_len):
    b = workloads.ragged(n, seed=seed, max_len=max_len, boundary_frac=0.05)
    return b


@pytest.mark.parametrize("indexed", [False, True])
def test_segments_match_whole_message_digests(hb, oracle_mod, indexed):
    b = _mixed_batch(3000, seed=71, max_len=20000)
    rng = np.random.default_rng(5)
    pieces, nrounds = _rounds(b, rng, max_pieces=6)
    got = _run_segmented(hb, b, pieces, nrounds, rng,
                         lambda a, p, o, l, s, out, si: hb.hash_batch_segments(a, p, o, l, s, out, si),
                         indexed=indexed)
    want = oracle_mod.hash_batch(None, b.packed, b.offsets, b.lengths, algs=b.algs)
    assert np.array_equal(got, want)


def test_segment_edge_cases(hb, oracle_mod):
    # zero-length middle pieces, a zero-length last piece after whole blocks,
    # a last piece of exactly 56/63/64 bytes (padding spills into a new block)
    lens = [0, 64, 128, 55 + 64, 56 + 128, 63 + 192, 64 * 5, 1000, 4096, 70000]
    b = workloads.scattered(lens, seed=72, overlap=False, mixed=True)
    cut_lists = [[0], [64, 0], [0, 64, 64, 0], [64, 55], [128, 56], [64, 0, 128, 63],
                 [64, 64, 64, 64, 64, 0], [960, 40], [4096, 0], [65536, 0, 4464]]
    pieces = [c for c in cut_lists]
    for c, L in zip(pieces, lens):
        assert sum(c) == L
    rng = np.random.default_rng(6)
    got = _run_segmented(hb, b, pieces, max(len(p) for p in pieces), rng,
                         lambda a, p, o, l, s, out, si: hb.hash_batch_segments(a, p, o, l, s, out, si),
                         indexed=True)
    want = oracle_mod.hash_batch(None, b.packed, b.offsets, b.lengths, algs=b.algs)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape", [0, 7, 10, 16, 18])
def test_segments_through_captured_plans(hb, oracle_mod, shape):
    b = _mixed_batch(2000, seed=73 + shape, max_len=9000)
    rng = np.random.default_rng(7 + shape)
    pieces, nrounds = _rounds(b, rng, max_pieces=4)
    max_n = b.n
    # fixed buffers for the graph: copy each round's arrays into them
    plan = hb.Plan(max_n, shape=shape, warps_per_sm=0)
    g_algs = torch.zeros(max_n, dtype=torch.uint8, device="cuda")
    g_off = torch.zeros(max_n, dtype=torch.int64, device="cuda")
    g_len = torch.zeros(max_n, dtype=torch.int32, device="cuda")
    g_seg = torch.zeros(max_n, dtype=torch.int64, device="cuda")
    g_out = torch.zeros((max_n, 32), dtype=torch.uint8, device="cuda")
    packed = torch.from_numpy(np.ascontiguousarray(b.packed)).cuda()
    plan.set_segments(g_seg)
    plan.capture(g_algs, packed, g_off, g_len, g_out)

    def call(a, p, o, l, s, out, si):
        m = a.numel()
        g_algs[:m] = a
        g_off[:m] = o
        g_len[:m] = l
        g_seg[:m] = s
        g_out[:m] = out
        plan.replay(m)
        out.copy_(g_out[:m])

    got = _run_segmented(hb, b, pieces, nrounds, rng, call)
    plan.close()
    want = oracle_mod.hash_batch(None, b.packed, b.offsets, b.lengths, algs=b.algs)
    assert np.array_equal(got, want)


def test_malformed_segment_is_skipped_and_reported(hb, oracle_mod):
    b = workloads.scattered([100, 200, 300], seed=74, overlap=False, mixed=True)
    packed, off, ln, algs = hb.to_device(b)
    hb.device_status()  # clear
    slots = torch.full((3, 32), 0x77, dtype=torch.uint8, device="cuda")
    # message 1 claims more pieces follow but 200 is not a multiple of 64
    seg = torch.from_numpy(hb.seg_words([0, 0, 0], [False, True, False])).cuda()
    hb.hash_batch_segments(algs, packed, off, ln, seg, slots)
    torch.cuda.synchronize()
    assert hb.device_status() & hb.DEV_SEGMENT
    got = slots.cpu().numpy()
    want = oracle_mod.hash_batch(None, b.packed, b.offsets, b.lengths, algs=b.algs)
    assert np.array_equal(got[[0, 2]], want[[0, 2]])
    assert (got[1] == 0x77).all()
