"""Host-side logic of the serving loop: arena bookkeeping and the admission /
batching policy.  No GPU needed."""
import numpy as np

from paper_2407_09333_b300.serve import ALIGN, Arena, Req, Scheduler, make_requests


def test_arena_first_fit_and_coalescing():
    a = Arena(10 * ALIGN)
    x = a.alloc(1)
    y = a.alloc(3 * ALIGN)
    z = a.alloc(ALIGN + 1)
    assert x == (0, ALIGN) and y == (ALIGN, 3 * ALIGN) and z == (4 * ALIGN, 2 * ALIGN)
    assert a.used == 6 * ALIGN
    assert a.alloc(5 * ALIGN) is None            # only 4 units left
    a.release(*y)
    assert a.alloc(5 * ALIGN) is None            # 7 units free, but as 3 + 4
    a.release(*x)                                # 0..4 coalesces into one range
    assert a.free[0] == (0, 4 * ALIGN)
    w = a.alloc(4 * ALIGN)
    assert w == (0, 4 * ALIGN)
    a.release(*w)
    a.release(*z)
    assert a.free == [(0, 10 * ALIGN)] and a.used == 0
    assert a.peak == 6 * ALIGN


def test_arena_random_alloc_free_keeps_invariants():
    rng = np.random.default_rng(0)
    a = Arena(1 << 20)
    live = []
    for _ in range(3000):
        if live and rng.random() < 0.45:
            a.release(*live.pop(int(rng.integers(len(live)))))
        else:
            got = a.alloc(int(rng.integers(1, 40000)))
            if got:
                live.append(got)
        # free list sorted, disjoint, coalesced; accounting consistent
        ends = [s + n for s, n in a.free]
        assert all(ends[k] < a.free[k + 1][0] for k in range(len(a.free) - 1))
        spans = sorted(live + a.free)
        assert all(spans[k][0] + spans[k][1] == spans[k + 1][0] for k in range(len(spans) - 1))
        assert a.used == sum(n for _, n in live)


def _req(rid, nbytes, nmsg=1):
    lens = np.full(nmsg, nbytes // nmsg, dtype=np.uint32)
    lens[0] += nbytes - int(lens.sum())
    return Req(rid, 0.0, 0, lens, [(0, nbytes)])


def test_scheduler_admits_in_order_under_budget_and_rejects_oversize():
    s = Scheduler(budget=10 * ALIGN, max_msgs=100, max_reqs=8)
    reqs = [_req(0, 4 * ALIGN), _req(1, 5 * ALIGN), _req(2, 3 * ALIGN), _req(3, 50 * ALIGN)]
    for r in reqs:
        s.arrive(r)
    assert s.admit(0.0) == 2                     # 4 + 5 fit, 3 does not
    assert [r.rid for r in s.ready] == [0, 1]
    batch = s.next_batch()
    assert [r.rid for r in batch] == [0, 1]
    s.finish(batch)
    assert s.admit(1.0) == 1                     # request 2 now fits; 3 is larger than the budget
    assert [r.rid for r in s.rejected] == [3]
    assert not s.waiting


def test_scheduler_batch_limits():
    s = Scheduler(budget=1 << 30, max_msgs=10, max_reqs=3)
    for k in range(6):
        s.arrive(_req(k, 1000, nmsg=4))
    s.admit(0.0)
    b1 = s.next_batch()
    assert len(b1) == 2                          # 4 + 4 messages; a third would exceed 10
    b2 = s.next_batch()
    assert len(b2) == 2
    assert len(s.next_batch()) == 2 and not s.ready


def test_request_payload_segments_cover_the_request():
    reqs = make_requests(200, 1000.0, seed=4, pool_bytes=1 << 20, max_len=1 << 16)
    for r in reqs:
        assert sum(n for _, n in r.segments) == r.nbytes
        assert all(off % 16 == 0 and off + n <= (1 << 20) for off, n in r.segments)
    arrivals = [r.arrival for r in reqs]
    assert arrivals == sorted(arrivals)
