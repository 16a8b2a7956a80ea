"""The serving loop on the GPU: every request's digests are the same as when
the request is hashed alone (and as the oracle's), whatever it was batched
with, including under a budget tight enough that admission has to wait."""
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


def _payload(req, pool_host):
    return np.concatenate([pool_host[o:o + n] for o, n in req.segments]) if req.segments else \
        np.zeros(0, dtype=np.uint8)


def _check_alone(api, oracle_mod, reqs, pool_host, oracle_every=7):
    for k, req in enumerate(reqs):
        assert req.done >= 0, req.rid
        payload = _payload(req, pool_host)
        buf = torch.from_numpy(np.concatenate([payload, np.zeros(16, np.uint8)])).cuda()
        off = torch.from_numpy(req.local_offsets.view(np.int64)).cuda()
        ln = torch.from_numpy(req.lengths.view(np.int32)).cuda()
        alone = api.hash_batch(req.alg, buf, off, ln).cpu().numpy()
        assert np.array_equal(req.digests, alone), req.rid
        if k % oracle_every == 0:
            want = oracle_mod.hash_batch(req.alg, payload, req.local_offsets, req.lengths)
            assert np.array_equal(req.digests, want), req.rid


def test_served_digests_equal_alone_digests(env, oracle_mod):
    api, serve, pool_host, pool_dev, pool_bytes = env
    reqs = serve.make_requests(150, 3000.0, seed=5, pool_bytes=pool_bytes, max_msgs=64,
                               max_len=1 << 16)
    srv = serve.Server(pool_dev, budget=512 << 20, slots=3, max_msgs=8192, max_reqs=64)
    srv.run(reqs, keep_digests=True)
    srv.close()
    assert srv.batched_reqs == len(reqs) and srv.batches < len(reqs)   # requests shared batches
    _check_alone(api, oracle_mod, reqs, pool_host)
    stats = serve.latency_stats(reqs)
    assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0


def test_tight_budget_makes_admission_wait(env, oracle_mod):
    api, serve, pool_host, pool_dev, pool_bytes = env
    reqs = serve.make_requests(60, 20000.0, seed=6, pool_bytes=pool_bytes, max_msgs=32,
                               max_len=1 << 15)
    biggest = max(r.nbytes for r in reqs)
    budget = max(4 * biggest, 1 << 20)
    srv = serve.Server(pool_dev, budget=budget, slots=2, max_msgs=4096, max_reqs=16)
    srv.run(reqs, keep_digests=True)
    srv.close()
    assert srv.sched.arena.peak <= srv.sched.arena.capacity
    assert any(r.admitted > r.arrival + 1e-4 for r in reqs)   # someone had to wait for space
    _check_alone(api, oracle_mod, reqs, pool_host, oracle_every=5)


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
