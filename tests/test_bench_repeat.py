"""bench.py's repetition rule (Section V): repeat the timed step until the Student-t 95 %
confidence half-width of its time is within a fraction of the mean (at least 3 runs, capped)."""
import math
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(steps=1, ci=0.0, cap=600.0):
    return types.SimpleNamespace(steps=steps, repeat_ci=ci, repeat_max_s=cap)


def _stepper(times):
    it = iter(times)
    return lambda: next(it)


@pytest.mark.parametrize("df,t", [(1, 12.7062), (2, 4.3027), (4, 2.7764), (9, 2.2622), (29, 2.0452)])
def test_t_quantiles_are_the_tabulated_student_values(df, t):
    # published two-sided 95 % points of Student's t
    assert bench.t975(df) == pytest.approx(t, abs=2e-3)


def test_fallback_table_is_conservative_and_decreasing():
    vals = [t for _, t in bench.T975]
    assert vals == sorted(vals, reverse=True)
    assert vals[-1] > 1.959964    # above the normal quantile


def test_ci95_closed_form():
    # xs = 1, 2, 3: mean 2, sample standard deviation 1, half-width t(0.975, 2) / sqrt(3)
    c = bench.ci95([1.0, 2.0, 3.0])
    assert c["n"] == 3 and c["mean_s"] == pytest.approx(2.0)
    assert c["half_width_s"] == pytest.approx(bench.t975(2) / math.sqrt(3.0))
    assert c["frac"] == pytest.approx(c["half_width_s"] / 2.0)
    assert bench.ci95([5.0]) is None
    assert bench.ci95([4.0, 4.0, 4.0])["half_width_s"] == 0.0


def test_exact_steps_without_the_rule():
    out, rep = bench.run_timed(_stepper([1.0, 2.0, 3.0, 4.0]), _args(steps=2), lambda x: x, world=1)
    assert out == [1.0, 2.0] and rep is None


def test_rule_stops_at_the_first_run_count_that_meets_the_precision():
    times = [1.10, 0.90, 1.05, 0.95, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0]
    out, rep = bench.run_timed(_stepper(times), _args(steps=1, ci=0.025), lambda x: x, world=1)
    n = len(out)
    assert n >= 3 and out == times[:n]
    assert rep["met"] and rep["frac"] <= 0.025 and rep["n"] == n
    # one run fewer did not meet it (the rule adds one run at a time)
    assert bench.ci95(times[:n - 1])["frac"] > 0.025


def test_rule_takes_at_least_three_runs():
    out, rep = bench.run_timed(_stepper([2.0, 2.0, 2.0, 2.0]), _args(steps=1, ci=0.025), lambda x: x, world=1)
    assert len(out) == 3 and rep["met"]


def test_rule_stops_at_the_time_cap():
    times = [1.0, 3.0] * 20
    out, rep = bench.run_timed(_stepper(times), _args(steps=1, ci=0.025, cap=10.0), lambda x: x, world=1)
    assert sum(out) >= 10.0 and sum(out[:-1]) < 10.0
    assert not rep["met"]


def test_rule_is_single_process():
    with pytest.raises(SystemExit):
        bench.run_timed(_stepper([1.0] * 5), _args(ci=0.025), lambda x: x, world=2)


def test_table_fallback_without_scipy(monkeypatch):
    monkeypatch.setitem(sys.modules, "scipy", None)     # import of scipy now fails
    assert bench.t975(4) == 2.776
    assert bench.t975(11) == 2.228                      # between entries: the smaller df's value
    assert bench.t975(500) == 1.980
