"""The autotuner's final round (host logic, no GPU): the setting in force
stays unless another candidate is clearly faster."""
import pytest

from paper_2407_09333_b300 import autotune


@pytest.fixture
def fake_timer(monkeypatch):
    # every launch of candidate k takes times[k] ms; make(k) returns k itself
    times = {}

    def fake_time_ms(torch, fn, reps):
        return times[fn]

    monkeypatch.setattr(autotune, "_time_ms", fake_time_ms)
    return times


def test_keeps_the_setting_in_force_within_the_margin(fake_timer):
    fake_timer.update({"a": 1.000, "b": 0.995, "keep": 1.000})
    first = {"a": 0.99, "b": 0.98, "keep": 1.00}
    assert autotune._final_round(None, first, lambda k: k, 3, keep="keep") == "keep"


def test_a_clearly_faster_candidate_wins(fake_timer):
    fake_timer.update({"a": 1.000, "b": 0.950, "keep": 1.000})
    first = {"a": 0.99, "b": 0.98, "keep": 1.00}
    assert autotune._final_round(None, first, lambda k: k, 3, keep="keep") == "b"


def test_the_setting_in_force_joins_the_final_even_when_slow_in_the_first_pass(fake_timer):
    # a lucky first pass put a, b and c ahead; timed again, none beats keep
    fake_timer.update({"a": 1.004, "b": 1.002, "c": 1.010, "keep": 1.000})
    first = {"a": 0.90, "b": 0.91, "c": 0.92, "keep": 1.00}
    assert autotune._final_round(None, first, lambda k: k, 3, keep="keep") == "keep"


def test_without_a_timed_setting_in_force_the_fastest_median_wins(fake_timer):
    fake_timer.update({"a": 1.004, "b": 1.002, "c": 1.010})
    first = {"a": 0.90, "b": 0.91, "c": 0.92}
    assert autotune._final_round(None, first, lambda k: k, 3, keep=("x", 8)) == "b"
    assert autotune._final_round(None, first, lambda k: k, 3) == "b"
