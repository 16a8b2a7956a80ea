"""The linear launch-cost model (host logic, no GPU)."""
import numpy as np
import pytest

from paper_2407_09333_b300 import costmodel


def test_work_counts_padded_blocks_times_ops():
    w = costmodel.work_by_alg([55, 56, 120], alg=2)
    assert list(w) == [0, 0, (1 + 2 + 3) * 1412]
    w = costmodel.work_by_alg([55, 56, 120], algs=np.array([0, 1, 0], np.uint8))
    assert list(w) == [(1 + 3) * 324, 2 * 613, 0]


def test_fit_recovers_rates_and_overhead():
    rng = np.random.default_rng(0)
    rate = np.array([2e-13, 3.5e-13, 7e-13])
    samples = []
    for _ in range(30):
        w = rng.uniform(0, 1e12, size=3) * (rng.random(3) < 0.7)
        samples.append((w, float(rate @ w + 1e-5)))
    m = costmodel.fit(samples)
    assert np.allclose(m.rate, rate, rtol=1e-6)
    assert m.overhead == pytest.approx(1e-5, rel=1e-4)
    assert m.r2 == pytest.approx(1.0)
    lens = np.full(1000, 16384)
    assert m.predict_batch(lens, alg=1) == pytest.approx(rate[1] * 1000 * 257 * 613 + 1e-5)


def test_fit_with_one_algorithm_only_and_noise():
    rng = np.random.default_rng(1)
    samples = [(np.array([0.0, 0.0, w]), 5e-13 * w + 2e-5 + rng.normal(0, 1e-7))
               for w in np.linspace(1e9, 1e12, 12)]
    m = costmodel.fit(samples)
    assert m.rate[0] == 0 and m.rate[1] == 0
    assert m.rate[2] == pytest.approx(5e-13, rel=1e-3)
    assert m.r2 > 0.999
    with pytest.raises(ValueError):
        costmodel.fit(samples[:1])
