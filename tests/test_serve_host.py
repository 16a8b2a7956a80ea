"""Host-side logic of the serving loop: ring and request-table bookkeeping
and the synthetic request stream.  No GPU needed."""
import numpy as np
import pytest

from paper_2407_09333_b300.serve import RingBook, device_bytes, make_requests


def test_ring_admits_in_order_until_full():
    b = RingBook(16, 4)
    assert b.admit(5) == (0, 0)
    assert b.admit(6) == (1, 5)
    assert not b.fits(6)            # 11 + 6 > 16
    assert b.fits(5)
    assert b.admit(5) == (2, 11)
    assert not b.fits(1)            # ring full
    assert b.tail - b.head == 16


def test_head_moves_only_past_finished_requests_in_order():
    b = RingBook(16, 8)
    r0, _ = b.admit(4)
    r1, _ = b.admit(4)
    r2, _ = b.admit(4)
    b.finish(r1)                    # out of order: r0 still holds the head
    assert (b.head, b.req_head) == (0, 0)
    b.finish(r0)                    # r0 and r1 leave together
    assert (b.head, b.req_head) == (8, 2)
    b.finish(r2)
    assert (b.head, b.req_head, b.tail) == (12, 3, 12)
    assert not b.open and not b.by_req


def test_request_table_limits_admission():
    b = RingBook(1024, 2)
    b.admit(1)
    b.admit(1)
    assert not b.fits(1)
    b.finish(0)
    assert b.fits(1)


def test_spans_split_at_the_wrap():
    b = RingBook(16, 4)
    assert b.spans(14, 5) == [(14, 0, 2), (0, 2, 3)]
    assert b.spans(3, 4) == [(3, 0, 4)]
    assert b.spans(16, 16) == [(0, 0, 16)]
    assert b.spans(30, 3, 8) == [(6, 0, 2), (0, 2, 1)]
    assert b.spans(5, 0) == []


def test_random_admit_finish_keeps_ring_invariants():
    rng = np.random.default_rng(0)
    b = RingBook(64, 8)
    live = []
    for _ in range(2000):
        if live and (rng.random() < 0.5 or not b.fits(8)):
            rc = live.pop(int(rng.integers(0, len(live))))
            b.finish(rc)
        else:
            m = int(rng.integers(1, 9))
            if b.fits(m):
                rc, first = b.admit(m)
                live.append(rc)
        assert 0 <= b.tail - b.head <= b.capacity
        assert 0 <= b.req_tail - b.req_head <= b.req_capacity
        # the head is the first message of the oldest unfinished request
        if b.open:
            assert b.open[0][1] == b.head
        else:
            assert b.head == b.tail


def test_rejects_non_power_of_two_capacity():
    with pytest.raises(ValueError):
        RingBook(100, 4)


def test_device_bytes_counts_ring_and_rounds():
    small = device_bytes(1 << 10, 16, 1, 1 << 10)
    assert device_bytes(1 << 11, 16, 1, 1 << 10) - small == (1 << 10) * 61
    assert device_bytes(1 << 10, 16, 2, 1 << 10) > small


def test_requests_are_seeded_and_messages_lie_inside_the_pool():
    pool = 1 << 24
    a = make_requests(40, 1000.0, seed=3, pool_bytes=pool, max_msgs=64, max_len=1 << 18)
    b = make_requests(40, 1000.0, seed=3, pool_bytes=pool, max_msgs=64, max_len=1 << 18)
    for x, y in zip(a, b):
        assert x.alg == y.alg and np.array_equal(x.lengths, y.lengths)
        assert np.array_equal(x.src, y.src)
        assert (x.src % 16 == 0).all()
        assert (x.src + x.lengths.astype(np.uint64) <= pool).all()
        assert 1 <= x.lengths.shape[0] <= 64 and x.alg in (0, 1, 2)
    arr = [r.arrival for r in a]
    assert arr == sorted(arr) and arr[0] >= 0


# ---------------------------------------------------------------------------
# admission by predicted completion time, under a fake clock

from paper_2407_09333_b300.serve import Admission, Req, prediction_stats  # noqa: E402


class _Model:
    """Cost model stand-in: work = bytes x per-byte rate of the algorithm,
    chain = longest message x per-byte chain rate."""
    RATE = (1e-12, 2e-12, 4e-12)        # s per byte, at full GPU throughput
    CHAIN = (2e-11, 3e-11, 6e-11)       # s per byte of one serial chain

    def work_seconds(self, lengths, alg):
        return float(np.asarray(lengths, dtype=np.float64).sum() * self.RATE[alg])

    def chain_time(self, lengths, alg):
        return float(np.asarray(lengths, dtype=np.float64).max(initial=0) * self.CHAIN[alg])

    def request_costs(self, lengths, alg):
        return self.work_seconds(lengths, alg), self.chain_time(lengths, alg)


def _requests(n, rate_per_s, seed):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for k in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        m = int(rng.integers(1, 50))
        lens = np.exp(rng.uniform(np.log(16), np.log(1 << 20), size=m)).astype(np.uint32)
        out.append(Req(k, t, int(rng.integers(0, 3)), lens, np.zeros(m, np.uint64)))
    return out


def _serve(adm, reqs):
    """Event-driven fake server: admitted work is done first come first
    served at adm.drain times the model's rate (req.work_s, which the policy
    sets at arrival, is already in served seconds); a request completes when
    its work is done, and not before its longest chain has run since
    admission.  Drives `adm` with the simulated clock; returns the order of
    admission."""
    import heapq
    pending, done_heap, order = [], [], []
    work_free = 0.0                        # when the FIFO server finishes the admitted work
    i = 0
    t = 0.0
    while i < len(reqs) or pending or done_heap:
        t_arr = reqs[i].arrival if i < len(reqs) else float("inf")
        t_done = done_heap[0][0] if done_heap else float("inf")
        if t_done <= t_arr:
            t, _, r = heapq.heappop(done_heap)
            r.done = t
            adm.finish(r, t)
        else:
            t, r = t_arr, reqs[i]
            i += 1
            if adm.arrive(r, t):
                pending.append(r)
        while pending and not adm.hold(t):
            r = pending.pop(0)
            r.admitted = t
            adm.admit(r, t)
            order.append(r.rid)
            work_free = max(work_free, t) + r.work_s
            heapq.heappush(done_heap, (max(work_free, t + r.chain_s) + adm.t0, r.rid, r))
    return order


@pytest.mark.parametrize("drain", [1.0, 0.8])
def test_admission_predicts_completion_of_a_first_come_first_served_device(drain):
    # the fake device serves admitted work at `drain` times the model's rate
    reqs = _requests(400, 2000.0 * drain, seed=1)
    adm = Admission(_Model(), t0=1e-4, drain=drain)
    order = _serve(adm, reqs)
    assert order == sorted(order)                       # admitted in arrival order
    for r in reqs:
        assert r.admitted == r.arrival                  # no cap: admitted on arrival
        assert r.done == pytest.approx(r.predicted_done, abs=1e-12)
    st = prediction_stats(reqs)
    assert st["requests"] == 400 and st["median_measured_over_predicted"] == pytest.approx(1.0)
    assert st["within_25pct"] == 1.0


def test_admission_holds_requests_while_the_backlog_exceeds_the_cap():
    reqs = _requests(600, 1e6, seed=2)                   # a burst: far above capacity
    cap = 2e-4
    seen = []

    class Watch(Admission):
        def admit(self, req, now):
            seen.append((self.backlog(now), self.inflight))
            super().admit(req, now)

    adm = Watch(_Model(), cap_s=cap)
    order = _serve(adm, reqs)
    assert order == sorted(order)
    assert all(b <= cap + 1e-12 or inflight == 0 for b, inflight in seen)
    assert any(r.admitted > r.arrival for r in reqs)    # some had to wait
    for r in reqs:                                      # predictions stay exact
        assert r.done == pytest.approx(r.predicted_done, abs=1e-12)


def test_admission_sheds_requests_predicted_past_the_target():
    model = _Model()
    probe = _requests(20000, 1.0, seed=3)
    mean_work = float(np.mean([model.work_seconds(r.lengths, r.alg) for r in probe]))
    load = 1.5                                          # offered load above capacity
    slo = 500 * mean_work
    plain = _requests(20000, load / mean_work, seed=3)
    _serve(Admission(model), plain)
    shed = _requests(20000, load / mean_work, seed=3)
    _serve(Admission(model, slo_s=slo), shed)
    lat_plain = np.array([r.done - r.arrival for r in plain])
    served = [r for r in shed if not r.rejected]
    lat_shed = np.array([r.done - r.arrival for r in served])
    assert np.percentile(lat_plain, 99) > 5 * slo       # unbounded queue without shedding
    assert lat_shed.max() <= slo + 1e-12                # every served request met the target
    # large requests are the first to miss the target, so what is shed is
    # about the excess work (1 - 1/load of it), in fewer requests
    shed_work = sum(r.work_s for r in shed if r.rejected) / sum(r.work_s for r in shed)
    assert 0.25 < shed_work < 0.45
    assert 0 < sum(r.rejected for r in shed) < len(shed) * shed_work
    assert all(r.done < 0 for r in shed if r.rejected)


def test_chain_factor_follows_a_slower_device():
    # the fake device runs every chain 1.6x longer than the model says: the
    # running factor converges there and later predictions come out right
    import heapq
    model = _Model()
    reqs = _requests(3000, 200.0, seed=5)              # light load: chain-bound requests
    adm = Admission(model, t0=1e-4, adapt=0.05)
    heap = []
    for r in reqs:
        while heap and heap[0][0] <= r.arrival:
            td, _, q = heapq.heappop(heap)
            q.done = td
            adm.finish(q, td)
        adm.arrive(r, r.arrival)
        adm.admit(r, r.arrival)
        r.admitted = r.arrival
        real = 1.6 * model.chain_time(r.lengths, r.alg)
        heapq.heappush(heap, (r.arrival + max(real, r.work_s) + adm.t0, r.rid, r))
    while heap:
        td, _, q = heapq.heappop(heap)
        q.done = td
        adm.finish(q, td)
    assert adm.chain_scale == pytest.approx(1.6, rel=0.05)
    late = [r for r in reqs[-500:] if r.chain_bound]
    ratio = np.array([(r.done - r.arrival) / (r.predicted_done - r.arrival) for r in late])
    assert np.median(ratio) == pytest.approx(1.0, abs=0.05)


def test_drain_is_calibrated_from_a_burst():
    from paper_2407_09333_b300.serve import calibrate_drain
    model = _Model()
    reqs = _requests(3000, 1e9, seed=4)                  # a burst: all at once
    for r in reqs:
        r.arrival = 0.0
    adm = Admission(model, drain=0.7)                    # the device's true rate
    _serve(adm, reqs)
    assert calibrate_drain(model, reqs) == pytest.approx(0.7, rel=0.1)


def test_admission_without_chain_calibration_uses_work_alone():
    from paper_2407_09333_b300 import costmodel
    m = costmodel.CostModel(np.array([1e-12, 2e-12, 3e-12]), 0.0, 1.0)
    assert m.chain_time([100, 5000], 2) == 0.0
    r = Req(0, 0.0, 2, [55, 56], [0, 0])
    adm = Admission(m)
    w, c = adm.estimate(r)
    assert w == pytest.approx(3e-12 * (1 + 2) * 1412) and c == 0.0
    # latency = 1 ms + ops / 2e7 for SM3 and ops / 5e7 for MD5: both recovered
    obs = [(2, L, 1e-3 + ((L + 72) // 64) * 1412 / 2e7) for L in (100, 5000, 16384, 70000)]
    obs += [(0, L, 1e-3 + ((L + 72) // 64) * 324 / 5e7) for L in (300, 9000, 120000)]
    m2 = costmodel.fit_chain(m, obs)
    assert m2.chain[2] == pytest.approx(2e7, rel=1e-6) and m2.chain[0] == pytest.approx(5e7, rel=1e-6)
    assert m2.chain[1] == 0 and m2.latency_t0 == pytest.approx(1e-3, rel=1e-6)
    assert m2.chain_time([100, 16384], 2) == pytest.approx(257 * 1412 / 2e7)


def test_request_costs_equal_work_seconds_and_chain_time():
    # the one-pass per-request estimate the admission policy uses equals the
    # model's general work and chain functions
    from paper_2407_09333_b300 import costmodel
    rng = np.random.Generator(np.random.PCG64(5))
    m = costmodel.CostModel(rate=np.array([7e-14, 5e-14, 4e-14]), overhead=3e-5, r2=1.0,
                            per_msg=np.array([2e-11, 0.0, 1e-11]),
                            chain=np.array([2.5e8, 3.1e8, 3.6e8]))
    for alg in (0, 1, 2):
        for n in (0, 1, 7, 4096):
            lens = rng.integers(0, 1 << 20, size=n).astype(np.uint32)
            work, chain = m.request_costs(lens, alg)
            assert work == pytest.approx(m.work_seconds(lens, alg), rel=1e-12, abs=0.0)
            assert chain == pytest.approx(m.chain_time(lens, alg), rel=1e-12, abs=0.0)
    nochain = costmodel.CostModel(rate=m.rate, overhead=m.overhead, r2=1.0, per_msg=m.per_msg)
    assert nochain.request_costs(np.array([100], np.uint32), 2)[1] == 0.0
