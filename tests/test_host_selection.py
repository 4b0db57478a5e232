"""Host-only checks of the timing estimator and the learned selection rule
(no GPU: a stand-in network supplies the predictions)."""
from __future__ import annotations

import numpy as np
import pytest

import sweep
from paper_1304_7053_gb300 import selector


def test_robust_mean_resolves_below_a_timer_step():
    """Times quantised to 1.024 us steps: a call of 16.9 us lands on 16.384
    or 17.408 us depending on its phase; the mean of the calls within 2 us of
    the median recovers the duration, the median snaps to a step, and a
    delayed call (+40 us) drops out."""
    step = 1.024e-3                      # ms
    true = 16.9e-3
    rng = np.random.default_rng(0)
    phase = rng.uniform(0.0, step, 4000)
    ts = list((np.floor((phase + true) / step) - np.floor(phase / step)) * step)
    ts.append(true + 0.040)
    med = sorted(ts)[len(ts) // 2]
    assert abs(med - true) > 0.4e-3
    assert sweep.robust_mean(ts) == pytest.approx(true, abs=0.03e-3)
    assert sweep.robust_mean([1.0, 1.0, 1.0]) == 1.0


def test_rule_keeps_default_unless_the_predicted_gain_clears_the_margin():
    pred = np.array([[1.0, 0.95, 2.0], [1.0, 0.7, 0.5], [1.0, 0.5, 0.1]])
    nv = np.array([3, 3, 1])
    dflt = np.array([0, 0, 0])
    # margin 0: the smallest prediction among the valid variants
    assert list(selector.rule_choice(pred, nv, np.zeros(3), dflt)) == [1, 2, 0]
    # margin 0.1: a 5% predicted gain is not enough, a 50% one is
    assert list(selector.rule_choice(pred, nv, np.full(3, 0.1), dflt)) == [0, 2, 0]
    # margin 1 never overrides; per-class margins apply row by row
    assert list(selector.rule_choice(pred, nv, np.ones(3), dflt)) == [0, 0, 0]
    assert list(selector.rule_choice(pred, nv, np.array([0.0, 1.0, 0.0]), dflt)) == [1, 0, 0]
    # the default need not be variant 0
    assert list(selector.rule_choice(pred, nv, np.full(3, 0.2), np.array([2, 1, 0]))) == [1, 2, 0]


def test_margins_are_picked_per_type_on_held_out_predictions():
    # type s: the predictions are right (variant 1 really is 30% faster);
    # type d: the network predicts a 5% gain for variant 1, which is really
    # 20% slower, and a 40% gain that is real
    times = np.array([[1.0, 0.7], [1.0, 0.7],          # s
                      [1.0, 1.2], [1.0, 0.6]])         # d
    pred = np.array([[1.0, 0.7], [1.0, 0.72],
                     [1.0, 0.95], [1.0, 0.6]])
    nv = np.array([2, 2, 2, 2])
    dflt = np.zeros(4, dtype=np.int64)
    m = selector.pick_margins(pred, times, nv, dflt, ["s", "s", "d", "d"])
    # s: every margin up to 0.2 takes both gains; ties go to the largest (0.2)
    assert m["s"] == 0.2
    # d: 0 and 0.02 take the bad switch; 0.05 .. 0.2 keep the default there
    # and still take the good one; the tie goes to 0.2
    assert m["d"] == 0.2
    # a network whose every switch loses: margin 1 (the default rule kept)
    bad = np.array([[1.0, 0.5], [1.0, 0.4]])
    m = selector.pick_margins(bad, np.array([[1.0, 1.1], [1.0, 1.3]]), np.array([2, 2]),
                              np.zeros(2, dtype=np.int64), ["z", "z"])
    assert m == {"z": 1.0}
    # row_margins spreads a type map over the classes
    assert list(selector.row_margins({"s": 0.1, "d": 1.0}, ["d", "s", "h"], 3)) == [1.0, 0.1, 0.0]
    assert list(selector.row_margins(0.05, None, 2)) == [0.05, 0.05]
