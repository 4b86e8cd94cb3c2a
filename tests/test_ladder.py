"""Ladder optimisation for uniform swap acceptance: the re-spacing rule pinned by closed forms
(CPU), the library's host logic against the oracle's independent version (CPU), and a full
optimisation driven by GPU runs against the same driven by oracle runs (GPU)."""
import math

import numpy as np
import pytest

import instances as I
from oracle import ladder as OL
from paper_2509_23043_gb300 import ladder as PL


def _acc_model(betas, sigma):
    """Acceptance of Gaussian energy laws with width sigma(beta_mid): erfc(dbeta sigma / 2)."""
    b = np.asarray(betas)
    mid = 0.5 * (b[1:] + b[:-1])
    return np.array([math.erfc((b[r + 1] - b[r]) * sigma(mid[r]) / 2) for r in range(len(b) - 1)])


@pytest.mark.parametrize("impl", ["oracle", "library"])
def test_constant_width_gives_equal_spacing_in_one_step(impl):
    b0 = I.geometric_betas(0.1, 3.0, 16)
    A = _acc_model(b0, lambda b: 7.0)
    att = np.full(15, 10 ** 12)
    acc = np.round(A * att).astype(np.int64)
    if impl == "oracle":
        new = np.array(OL.respace(list(b0), OL.distances(acc, att)))
    else:
        new = PL.respace(b0, PL.pair_distance(acc, att))
    assert np.allclose(new, np.linspace(0.1, 3.0, 16), atol=1e-9)


def test_equal_acceptance_is_a_fixed_point_and_ends_stay():
    b0 = np.array([0.2, 0.5, 0.7, 1.4, 2.0])
    acc, att = np.full(4, 300), np.full(4, 1000)
    for new in (np.array(OL.respace(list(b0), OL.distances(acc, att))),
                PL.respace(b0, PL.pair_distance(acc, att))):
        # equal distances per pair: the new ladder re-spaces D uniformly, which for equal d
        # returns the old points
        assert np.allclose(new, b0, atol=1e-12)


def test_library_and_oracle_rules_agree_and_stay_monotone():
    g = np.random.default_rng(8)
    for _ in range(20):
        R = int(g.integers(3, 40))
        b0 = np.sort(g.uniform(0.05, 5.0, R))
        att = g.integers(1, 5000, R - 1)
        acc = (att * g.uniform(0, 1, R - 1)).astype(np.int64)
        a = np.array(OL.respace(list(b0), OL.distances(acc, att)))
        b = PL.respace(b0, PL.pair_distance(acc, att))
        assert np.allclose(a, b, rtol=0, atol=1e-9)
        assert a[0] == b0[0] and a[-1] == b0[-1] and np.all(np.diff(a) >= 0)


def test_width_growing_with_beta_puts_points_where_the_integral_says():
    # sigma(beta) = c beta: the distance from beta_min is c (beta^2 - beta_min^2) / 2, so the
    # fixed point ladder is beta_k = sqrt(beta_min^2 + k/(R-1) (beta_max^2 - beta_min^2));
    # iterating the rule from a geometric ladder approaches it
    R, lo, hi = 12, 0.2, 3.0
    target = np.sqrt(lo ** 2 + np.arange(R) / (R - 1) * (hi ** 2 - lo ** 2))
    b = I.geometric_betas(lo, hi, R)
    for _ in range(25):
        A = _acc_model(b, lambda x: 3.0 * x)
        att = np.full(R - 1, 10 ** 12)
        b = PL.respace(b, PL.pair_distance(np.round(A * att), att))
    assert np.allclose(b, target, atol=2e-3)


@pytest.mark.gpu
def test_ladder_optimisation_on_gpu_matches_oracle_driven():
    insts = [I.ea_instance(4, index=40 + k) for k in range(3)]
    b0 = I.geometric_betas(0.1, 3.0, 8)
    lg, hg = PL.optimise_ladder(insts, b0, iterations=3, sweeps=300, seed=0x1ADD)
    lo, ho = OL.optimise_ladder(insts, b0, iterations=3, sweeps=300, seed=0x1ADD)
    for a, b in zip(hg, ho):
        assert np.allclose(a["betas"], b["betas"], atol=1e-9)
        assert np.allclose(a["acceptance"], np.array(b["accepted"]) / np.array(b["attempted"]),
                           atol=0)
    assert np.allclose(lg, lo, atol=1e-9)
