"""The streaming serving path on the GPU.

A round claims ready messages of a ring, hashes their next segments and
advances them; the server drives rounds on several streams.  Every message's
final slot must equal the CPU oracle's digest of the whole message (and the
plain single-algorithm path's), whatever segments, rounds and batch-mates it
had, including when the ring is small enough that admission waits and
entries are reused.
"""
import numpy as np
import pytest

from paper_2407_09333_b300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09333_b300 import api, build, serve
    build.build()
    api.lib()
    pool_bytes = 32 << 20
    pool_host = workloads.fixed(1, pool_bytes, seed=77).packed
    pool_dev = torch.from_numpy(np.ascontiguousarray(pool_host)).cuda()
    return api, serve, pool_host, pool_dev, pool_bytes


def _ring(api, cap, req_cap):
    dev = "cuda"
    return {
        "src": torch.zeros(cap, dtype=torch.int64, device=dev),
        "prior": torch.zeros(cap, dtype=torch.int64, device=dev),
        "len": torch.zeros(cap, dtype=torch.int32, device=dev),
        "req": torch.zeros(cap, dtype=torch.int32, device=dev),
        "alg": torch.zeros(cap, dtype=torch.uint8, device=dev),
        "state": torch.zeros(cap, dtype=torch.int32, device=dev),
        "slots": torch.zeros((cap, 32), dtype=torch.uint8, device=dev),
        "req_remaining": torch.zeros(req_cap, dtype=torch.int32, device=dev),
        "req_done": torch.zeros(req_cap, dtype=torch.int32).pin_memory(),
    }


@pytest.mark.parametrize("in_place", [False, True])
def test_rounds_hash_a_ring_segment_by_segment(env, oracle_mod, in_place):
    api, serve, pool_host, pool_dev, pool_bytes = env
    n, per_req = 700, 10
    b = workloads.ragged(n, seed=81, max_len=9000, boundary_frac=0.05)
    cap, nreq = 1024, (n + per_req - 1) // per_req
    ring = _ring(api, cap, 128)
    packed = torch.from_numpy(np.ascontiguousarray(b.packed)).cuda()
    base = packed.data_ptr()
    ring["src"][:n] = torch.from_numpy((b.offsets.astype(np.int64) + base)).cuda()
    ring["len"][:n] = torch.from_numpy(b.lengths.view(np.int32)).cuda()
    ring["alg"][:n] = torch.from_numpy(b.algs).cuda()
    req = np.arange(n, dtype=np.int32) // per_req
    ring["req"][:n] = torch.from_numpy(req).cuda()
    ring["req_remaining"][:nreq] = torch.from_numpy(np.bincount(req).astype(np.int32)).cuda()
    ring["state"][:n] = api.RING_READY
    staging = torch.empty(64 << 10, dtype=torch.uint8, device="cuda")
    seg = 512
    rounds = [api.Round(ring, 300, None if in_place else staging[i * (32 << 10):], 32 << 10, seg,
                        shape=16) for i in range(2)]
    streams = [torch.cuda.Stream() for _ in rounds]
    torch.cuda.synchronize()
    expect = int(sum(max(1, -(-int(L) // seg)) for L in b.lengths))
    claimed = 0
    for it in range(2000):
        for r, s in zip(rounds, streams):
            r.launch(0, n, stream=s)
        torch.cuda.synchronize()
        claimed += sum(r.report()[0] for r in rounds)
        if (ring["req_done"].numpy()[:nreq] == 1).all():
            break
    assert (ring["req_done"].numpy()[:nreq] == 1).all()
    assert claimed == expect                       # every segment exactly once
    assert (ring["state"][:n] == api.RING_FREE).all()
    assert (ring["req_remaining"][:nreq] == 0).all()
    assert (ring["prior"][:n].cpu().numpy() == b.lengths.astype(np.int64)).all()
    want = oracle_mod.hash_batch(None, b.packed, b.offsets, b.lengths, algs=b.algs)
    assert np.array_equal(ring["slots"][:n].cpu().numpy(), want)
    assert api.device_status() == 0
    for r in rounds:
        r.close()


def test_round_reports_a_request_index_outside_the_table(env, oracle_mod):
    api = env[0]
    b = workloads.fixed(40, 300, seed=83)
    ring = _ring(api, 64, 4)
    packed = torch.from_numpy(np.ascontiguousarray(b.packed)).cuda()
    ring["src"][:40] = torch.from_numpy(b.offsets.astype(np.int64) + packed.data_ptr()).cuda()
    ring["len"][:40] = torch.from_numpy(b.lengths.view(np.int32)).cuda()
    ring["alg"][:40] = 2
    req = np.zeros(40, dtype=np.int32)
    req[7] = 1000                                     # outside the 4-entry request table
    ring["req"][:40] = torch.from_numpy(req).cuda()
    ring["req_remaining"][0] = 39
    ring["state"][:40] = api.RING_READY
    api.device_status()
    r = api.Round(ring, 64, None, 1 << 20, 4096, shape=16)
    s = torch.cuda.Stream()
    r.launch(0, 40, stream=s)
    torch.cuda.synchronize()
    assert api.device_status() & api.DEV_BOUNDS
    assert int(ring["req_remaining"][0].item()) == 0 and ring["req_done"][0].item() == 1
    want = oracle_mod.hash_batch(2, b.packed, b.offsets, b.lengths)
    assert np.array_equal(ring["slots"][:40].cpu().numpy(), want)   # every digest still written
    r.close()


def test_round_arguments_are_checked(env):
    api = env[0]
    ring = _ring(api, 64, 4)
    staging = torch.empty(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.HashBatchError) as e:
        api.Round(ring, 16, staging, 4096, 100)        # segment not a multiple of 64
    assert e.value.code == -10
    bad = dict(ring, state=torch.zeros(48, dtype=torch.int32, device="cuda"))
    with pytest.raises(api.HashBatchError):
        api.Round(bad, 16, staging, 4096, 128)          # capacity not a power of two
    with pytest.raises(ValueError):                    # flags must be host memory
        api.Round(dict(ring, req_done=torch.zeros(4, dtype=torch.int32, device="cuda")),
                  16, staging, 4096, 128)
    r = api.Round(ring, 16, staging, 4096, 128)
    r.close()


def _check_requests(api, oracle_mod, reqs, pool_host, oracle_every=3):
    for k, req in enumerate(reqs):
        assert req.done >= 0, req.rid
        m = req.lengths.shape[0]
        if m == 0:
            continue
        offs = req.src
        if k % oracle_every == 0:
            want = oracle_mod.hash_batch(req.alg, pool_host, offs, req.lengths)
            assert np.array_equal(req.digests, want), req.rid
        # the plain single-algorithm path on the same bytes
        if k % (2 * oracle_every) == 1:
            buf = torch.from_numpy(np.ascontiguousarray(pool_host)).cuda()
            alone = api.hash_batch(req.alg, buf, torch.from_numpy(offs.view(np.int64)).cuda(),
                                   torch.from_numpy(req.lengths.view(np.int32)).cuda())
            assert np.array_equal(req.digests, alone[:m].cpu().numpy()), req.rid


def test_served_through_staging_digests_equal_oracle(env, oracle_mod):
    api, serve, pool_host, pool_dev, pool_bytes = env
    reqs = serve.make_requests(120, 3000.0, seed=5, pool_bytes=pool_bytes, max_msgs=64,
                               max_len=1 << 16)
    srv = serve.Server(pool_dev, budget=256 << 20, rounds=3, segment_bytes=4096,
                       max_msgs=4096, capacity=1 << 14, req_capacity=256, shape=16,
                       warps_per_sm=8, in_place=False)
    srv.run(reqs, keep_digests=True)
    srv.close()
    assert srv.staging is not None
    assert srv.segments > sum(r.lengths.shape[0] for r in reqs)   # long messages were cut
    _check_requests(api, oracle_mod, reqs, pool_host)
    stats = serve.latency_stats(reqs)
    assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert api.device_status() == 0


def test_served_in_place_digests_equal_oracle(env, oracle_mod):
    api, serve, pool_host, pool_dev, pool_bytes = env
    reqs = serve.make_requests(60, 3000.0, seed=9, pool_bytes=pool_bytes, max_msgs=64,
                               max_len=1 << 16)
    # a request without messages finishes on arrival
    reqs.insert(5, serve.Req(10 ** 6, reqs[5].arrival, 1, [], []))
    srv = serve.Server(pool_dev, budget=128 << 20, rounds=2, segment_bytes=(12288, 8192, 4096),
                       max_msgs=4096, capacity=1 << 14, req_capacity=256, in_place=True)
    srv.run(reqs, keep_digests=True)
    srv.close()
    assert srv.staging is None
    assert reqs[5].done >= 0 and reqs[5].digests.shape == (0, 32)
    _check_requests(api, oracle_mod, reqs, pool_host, oracle_every=2)


def test_small_ring_makes_admission_wait_and_reuses_entries(env, oracle_mod):
    api, serve, pool_host, pool_dev, pool_bytes = env
    reqs = serve.make_requests(80, 50000.0, seed=6, pool_bytes=pool_bytes, max_msgs=32,
                               max_len=1 << 15)
    srv = serve.Server(pool_dev, budget=64 << 20, rounds=2, segment_bytes=2048,
                       max_msgs=512, capacity=128, req_capacity=8, shape=14, warps_per_sm=8)
    srv.run(reqs, keep_digests=True)
    srv.close()
    assert srv.book.tail > srv.book.capacity                      # the ring wrapped
    assert any(r.admitted > r.arrival + 1e-4 for r in reqs)       # someone had to wait
    _check_requests(api, oracle_mod, reqs, pool_host, oracle_every=2)


@pytest.fixture(scope="module")
def big_pool(env):
    # room for 1 MiB messages at any byte offset
    pool_bytes = 256 << 20
    pool_host = workloads.fixed(1, pool_bytes, seed=78).packed
    pool_dev = torch.from_numpy(np.ascontiguousarray(pool_host)).cuda()
    yield pool_host, pool_dev, pool_bytes
    del pool_dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("in_place", [True, False])
def test_served_at_config5_shape_unaligned_equals_oracle(env, big_pool, oracle_mod, in_place):
    # The serving workload's own request shape: 1-4096 messages per request
    # (log-uniform count), lengths log-uniform in [16 B, 1 MiB], one random
    # algorithm per request, every message at a random byte offset of the
    # clients' pool; served by the benchmark's server (8 GiB budget, two
    # rounds, default segments), arrivals overlapping.  Every digest of every
    # request is compared with the ragged path run once over all messages,
    # and a sample of each request (first, last, longest and five seeded
    # messages) with the oracle.
    api, serve = env[0], env[1]
    pool_host, pool_dev, pool_bytes = big_pool
    reqs = serve.make_requests(200, 2000.0, seed=91 + int(in_place), pool_bytes=pool_bytes,
                               align=1)
    assert max(r.lengths.shape[0] for r in reqs) > 1000
    assert max(int(r.lengths.max()) for r in reqs) > (1 << 19)
    assert sum(int((r.src % 16 != 0).sum()) for r in reqs) > 0
    srv = serve.Server(pool_dev, in_place=in_place)
    srv.run(reqs, keep_digests=True)
    srv.close()
    assert srv.segments > sum(r.lengths.shape[0] for r in reqs)   # long messages were cut
    assert all(r.done >= 0 for r in reqs)
    got = np.concatenate([r.digests for r in reqs])
    src = np.concatenate([r.src for r in reqs])
    lens = np.concatenate([r.lengths for r in reqs])
    algs = np.concatenate([np.full(r.lengths.shape[0], r.alg, np.uint8) for r in reqs])
    alone = api.hash_batch_mixed(torch.from_numpy(algs).cuda(), pool_dev,
                                 torch.from_numpy(src.view(np.int64)).cuda(),
                                 torch.from_numpy(lens.view(np.int32)).cuda()).cpu().numpy()
    bad = np.nonzero((got != alone).any(axis=1))[0]
    assert bad.size == 0, "%d of %d served digests differ from the ragged path" % (bad.size, len(got))
    rng = np.random.default_rng(92)
    pick, base = [], 0
    for r in reqs:
        m = r.lengths.shape[0]
        pick += [base, base + m - 1, base + int(np.argmax(r.lengths))]
        pick += (base + rng.integers(0, m, size=5)).tolist()
        base += m
    pick = np.unique(np.array(pick, dtype=np.int64))
    want = oracle_mod.hash_batch(None, pool_host, src[pick], lens[pick], algs=algs[pick],
                                 threads=oracle_mod.host_threads())
    bad = np.nonzero((got[pick] != want).any(axis=1))[0]
    assert bad.size == 0, "%d of %d sampled digests differ from the oracle" % (bad.size, len(pick))
    assert api.device_status() == 0


def test_served_from_host_memory_equals_oracle(env, oracle_mod):
    # host ingress: the clients' bytes stay in pinned host memory and each
    # round's copy step brings its segments over the bus, at any byte offset
    api, serve, pool_host, pool_dev, pool_bytes = env
    host_pool = torch.from_numpy(np.ascontiguousarray(pool_host)).pin_memory()
    reqs = serve.make_requests(80, 4000.0, seed=13, pool_bytes=pool_bytes, max_msgs=64,
                               max_len=1 << 17, align=1)
    srv = serve.Server(host_pool, budget=128 << 20, rounds=2, segment_bytes=(12288, 8192, 4096),
                       max_msgs=4096, capacity=1 << 14, req_capacity=256, in_place=False)
    assert srv.host_ingress
    srv.run(reqs, keep_digests=True)
    srv.close()
    _check_requests(api, oracle_mod, reqs, pool_host, oracle_every=1)
    assert api.device_status() == 0
    with pytest.raises(ValueError):
        serve.Server(host_pool, budget=128 << 20, in_place=True)


def test_served_under_admission_policy_equals_oracle(env, oracle_mod):
    # the live server with the admission policy: a tight hold cap makes
    # requests wait on the host, every admitted request gets a predicted
    # completion time, and the digests are those of the oracle; a target of
    # zero sheds every request at arrival and nothing reaches the device
    api, serve, pool_host, pool_dev, pool_bytes = env
    from paper_2407_09333_b300 import costmodel
    model = costmodel.fit_chain(
        costmodel.CostModel(np.array([1e-13, 1e-13, 1e-13]), 0.0, 1.0),
        [(a, 1 << 16, 2e-3) for a in (0, 1, 2)])
    reqs = serve.make_requests(90, 20000.0, seed=15, pool_bytes=pool_bytes, max_msgs=64,
                               max_len=1 << 16, align=1)
    srv = serve.Server(pool_dev, budget=128 << 20, rounds=2, segment_bytes=(12288, 8192, 4096),
                       max_msgs=4096, capacity=1 << 14, req_capacity=256, in_place=True)
    adm = serve.Admission(model, cap_s=1e-6, drain=0.9)
    srv.run(reqs, keep_digests=True, admission=adm)
    assert all(r.predicted_done >= r.admitted >= r.arrival for r in reqs)
    assert any(r.admitted > r.arrival + 1e-4 for r in reqs)        # the cap held some back
    _check_requests(api, oracle_mod, reqs, pool_host, oracle_every=1)
    assert adm.inflight == 0
    shed = serve.make_requests(30, 20000.0, seed=16, pool_bytes=pool_bytes, max_msgs=64,
                               max_len=1 << 16)
    segments = srv.segments
    srv.run(shed, admission=serve.Admission(model, slo_s=0.0))
    srv.close()
    assert all(r.rejected and r.done < 0 for r in shed)
    assert srv.segments == segments                                 # nothing was hashed
    assert api.device_status() == 0


def test_completion_flags_must_be_mapped_host_memory(env):
    api = env[0]
    plan = api.Plan(64)
    d = torch.zeros(64, dtype=torch.int32, device="cuda")
    p = api.ctypes.c_void_p(d.data_ptr())
    # device memory where host flags are expected: rejected, nothing launched
    assert api.lib().hash_plan_set_completion(plan._h, p, p, p) == -10
    pinned = torch.zeros(64, dtype=torch.int32).pin_memory()
    plan.set_completion(d, d, pinned)
    plan.close()
