"""Time to solution of Supplementary S5, pinned by its closed form."""
import math

import numpy as np
import pytest

from paper_2509_23043_gb300 import tts


def test_repetitions_closed_form():
    # R = ceil(log(0.01) / log(1 - s))
    assert tts.repetitions(0.5) == 7          # log(0.01)/log(0.5) = 6.64
    assert tts.repetitions(0.99) == 1
    assert tts.repetitions(0.9) == 2          # 0.1^2 = 0.01
    assert tts.repetitions(0.1) == 44         # log(0.01)/log(0.9) = 43.7
    assert tts.repetitions(1.0) == 1
    assert math.isinf(tts.repetitions(0.0))
    # the defining property: R runs reach the target, R - 1 do not
    for s in np.linspace(0.01, 0.98, 50):
        R = tts.repetitions(float(s))
        assert 1 - (1 - s) ** R >= 0.99 - 1e-12
        if R > 1:
            assert 1 - (1 - s) ** (R - 1) < 0.99


def test_optimal_tts_takes_the_minimum_over_run_lengths():
    t = [100, 200, 400, 800]
    s = [0.05, 0.3, 0.5, 0.6]
    vals = [tts.tts_sweeps(a, b) for a, b in zip(t, s)]
    best, ta = tts.optimal_tts(t, s)
    assert best == min(vals) and ta == t[int(np.argmin(vals))]


def test_success_curve_from_first_success_sweeps():
    solved = np.array([-1, 50, 100, 250, 400, -1])
    assert tts.success_curve(solved, [50, 100, 300, 500]) == pytest.approx([1 / 6, 2 / 6, 3 / 6, 4 / 6])


def test_fit_exponent_recovers_an_exact_exponential_and_the_two_point_slope():
    n = [16, 18, 20, 22, 24]
    A, k = 3.5, 0.846
    fit = tts.fit_exponent(n, [A * math.exp(k * x) for x in n])
    assert fit[0] == pytest.approx(A, rel=1e-9) and fit[1] == pytest.approx(k, rel=1e-12)
    # two sizes: the slope of the line through both points
    a, b = tts.fit_exponent([16, 20], [1000.0, 9000.0])
    assert b == pytest.approx(math.log(9.0) / 4) and a * math.exp(16 * b) == pytest.approx(1000.0)
    # infinite or missing sizes are left out; fewer than two finite sizes give no fit
    assert tts.fit_exponent([16, 18, 20], [100.0, math.inf, 100.0 * math.exp(4 * 0.5)])[1] == \
        pytest.approx(0.5)
    assert tts.fit_exponent([16, 18], [100.0, math.inf]) is None

