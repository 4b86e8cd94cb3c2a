"""Time to solution at a target success probability (Supplementary S5).

With success probability s for one run of t_a sweeps, R independent runs all fail with
probability (1 - s)^R, so reaching success probability P_target needs
R = ceil(log(1 - P_target) / log(1 - s)) runs. The time to solution in sweeps is
TTS(t_a) = t_a * R. The reported value is its minimum over the run lengths tried, and a
measured time per sweep converts it to seconds.
"""
from __future__ import annotations

import math

import numpy as np

P_TARGET = 0.99


def repetitions(s: float, p_target: float = P_TARGET) -> float:
    """R(P_target) for a per-run success probability s (inf when s = 0, 1 when s = 1)."""
    if s <= 0.0:
        return math.inf
    if s >= 1.0:
        return 1.0
    return float(math.ceil(math.log(1.0 - p_target) / math.log(1.0 - s)))


def tts_sweeps(t_a: float, s: float, p_target: float = P_TARGET) -> float:
    """TTS in sweeps for run length t_a with success probability s(t_a)."""
    return t_a * repetitions(s, p_target)


def optimal_tts(run_lengths, successes, p_target: float = P_TARGET) -> tuple[float, float]:
    """(min over t_a of TTS(t_a), the minimising t_a) from s(t_a) at the given run lengths."""
    vals = [tts_sweeps(t, s, p_target) for t, s in zip(run_lengths, successes)]
    k = int(np.argmin(vals))
    return vals[k], float(run_lengths[k])


def success_curve(solved_at: np.ndarray, run_lengths) -> list[float]:
    """s(t_a) from the sweep at which each independent run first succeeded (-1: never)."""
    solved_at = np.asarray(solved_at)
    return [float(np.mean((solved_at >= 0) & (solved_at <= t))) for t in run_lengths]


def fit_exponent(sizes, tts) -> tuple[float, float] | None:
    """(A, k) of TTS(n) = A exp(k n), least squares on log TTS against n (Fig. 5, S5). None
    when fewer than two sizes have a finite, positive TTS."""
    n = np.asarray(sizes, dtype=np.float64)
    t = np.asarray(tts, dtype=np.float64)
    ok = np.isfinite(t) & (t > 0)
    if ok.sum() < 2:
        return None
    k, log_a = np.polyfit(n[ok], np.log(t[ok]), 1)
    return float(np.exp(log_a)), float(k)
