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
