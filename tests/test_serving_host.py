"""Host side of the serving workload (CPU): the open-loop Poisson request schedule."""
import math

import numpy as np

from paper_2512_16543_gb300 import serving


def test_poisson_schedule_rate_order_and_states():
    rate, dur, n_states = 50_000.0, 0.5, 2000
    sched = serving.poisson_schedule(rate, dur, n_states, seed=7)
    assert sched == serving.poisson_schedule(rate, dur, n_states, seed=7)     # seeded
    assert sched != serving.poisson_schedule(rate, dur, n_states, seed=8)
    t = np.array([a for a, _ in sched])
    s = np.array([b for _, b in sched])
    mean = rate * dur
    assert abs(len(sched) - mean) < 5 * math.sqrt(mean)          # Poisson count, 5 sigma
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] < dur
    gaps = np.diff(t)
    assert abs(gaps.mean() * rate - 1.0) < 5 / math.sqrt(len(gaps))   # exponential gaps
    assert abs(gaps.std() * rate - 1.0) < 0.05                    # exponential: std = mean
    assert s.min() >= 0 and s.max() < n_states
    counts = np.bincount(s, minlength=n_states)                  # uniform over the states
    expect = len(s) / n_states
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < n_states + 6 * math.sqrt(2 * n_states)


def test_poisson_schedule_small_and_empty():
    assert serving.poisson_schedule(1000.0, 0.0, 4, seed=1) == []
    sched = serving.poisson_schedule(10.0, 1.0, 3, seed=3)
    assert all(0 <= a < 1.0 and 0 <= b < 3 for a, b in sched)
