"""A batch dominated by a few giant messages.

Each message is one serial chain of compressions (RFC 1321 Sec. 3.4,
FIPS 180-4 Sec. 6.1.2, GB/T 32905 Sec. 5.3), so a giant message takes as
long as its chain whatever else runs.  The ragged path starts the longest
messages first and completes the rest of the batch around them; with
per-request completion flags the caller can take the small messages'
digests while the giant chains still run.
"""
import time

import numpy as np
import pytest

from paper_2407_09333_b300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GIANT = 24 << 20


def test_small_messages_complete_while_giant_chains_run(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09333_b300 import api, build
    build.build()
    rng = np.random.default_rng(61)
    n_small = 20000
    lens = np.concatenate([np.full(4, GIANT), rng.integers(0, 2000, n_small)]).astype(np.uint32)
    algs = np.concatenate([[2, 2, 1, 0], rng.integers(0, 3, n_small)]).astype(np.uint8)
    b = workloads.scattered(lens, seed=62, overlap=False)
    b = workloads.Batch(b.packed, b.offsets, b.lengths, algs)
    n = b.n
    packed, off, ln, algs_d = api.to_device(b)
    # request 0: the small messages; request 1: the four giant ones
    msg_req = torch.tensor(np.r_[np.ones(4), np.zeros(n_small)].astype(np.int32), device="cuda")
    remaining = torch.tensor([n_small, 4], dtype=torch.int32, device="cuda")
    done = torch.zeros(2, dtype=torch.int32).pin_memory()
    out = torch.zeros((n, 32), dtype=torch.uint8, device="cuda")
    plan = api.Plan(n)
    try:
        plan.set_completion(msg_req, remaining, done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.run(algs_d, packed, off, ln, out)
        small_at = giant_at = None
        giant_seen_with_small = None
        while time.perf_counter() - t0 < 120:
            flags = done.tolist()
            if small_at is None and flags[0]:
                small_at = time.perf_counter() - t0
                giant_seen_with_small = flags[1]
            if flags[1]:
                giant_at = time.perf_counter() - t0
                break
            time.sleep(1e-4)
        torch.cuda.synchronize()
    finally:
        plan.close()
    assert small_at is not None and giant_at is not None, (small_at, giant_at)
    # the small messages were done, and flagged, while the giant chains ran
    assert giant_seen_with_small == 0
    assert giant_at > 4 * small_at, (small_at, giant_at)
    print("small messages done at %.1f ms; giant chains (%d MiB) at %.1f ms: %.0f MB/s per chain"
          % (1e3 * small_at, GIANT >> 20, 1e3 * giant_at, GIANT / giant_at / 1e6))
    got = out.cpu().numpy()
    sel = np.r_[np.arange(4), 4 + np.arange(0, n_small, 13)]
    want = oracle_mod.hash_batch(None, b.packed, b.offsets[sel], b.lengths[sel], algs=algs[sel],
                                 threads=oracle_mod.host_threads())
    assert np.array_equal(got[sel], want)
