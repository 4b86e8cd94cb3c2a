"""Temperature-ladder optimisation for uniform swap acceptance (Methods, parallel tempering).

The paper fixes, per problem family and size, a ladder whose neighbouring slots swap with
about equal probability, found by an adaptive procedure it cites but does not spell out. The
procedure here is iterative and uses the library's own swap statistics:
1. Run PT on a set of instances with the current ladder.
2. Read the accepted/attempted swap counts of every pair.
3. Re-space the inverse temperatures so that every pair carries the same share of a
   "thermodynamic distance". The ends stay fixed.

Distance of a pair. For Gaussian energy laws of width sigma at neighbouring slots, a swap is
accepted with probability erfc(dbeta * sigma / 2). So d_r = 2 erfcinv(A_r) estimates
dbeta_r * sigma, which is additive along the ladder. With D(beta) the piecewise-linear
cumulative distance through the current ladder points, the new point k solves
D(beta_k) = k / (R - 1) * D(beta_max). A ladder whose pairs already have equal acceptance is a
fixed point.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfcinv

from . import Config, create_instances, destroy, read_stats, run_cycles

A_MIN, A_MAX = 1e-4, 1.0 - 1e-9


def pair_distance(accepted: np.ndarray, attempted: np.ndarray) -> np.ndarray:
    """d_r = 2 erfcinv(A_r) with A_r clipped to [1e-4, 1 - 1e-9]."""
    A = np.clip(np.asarray(accepted, np.float64) / np.maximum(np.asarray(attempted, np.float64), 1.0),
                A_MIN, A_MAX)
    return 2.0 * erfcinv(A)


def respace(betas: np.ndarray, d: np.ndarray) -> np.ndarray:
    """New ladder with equal distance per pair, by inverting the piecewise-linear D(beta)."""
    betas = np.asarray(betas, np.float64)
    D = np.concatenate([[0.0], np.cumsum(d)])
    R = len(betas)
    targets = D[-1] * np.arange(R) / (R - 1)
    out = np.interp(targets, D, betas)
    out[0], out[-1] = betas[0], betas[-1]
    return out


def optimise_ladder(instances, betas0, iterations: int = 5, sweeps: int = 2000,
                    update: int = 0, seed: int = 0x1ADD, stream=None):
    """Run `iterations` rounds of (PT for `sweeps` sweeps on every instance, re-space). All
    instances share one ladder, as in the paper. Returns (ladder, history), where history
    holds each round's ladder and per-pair acceptance."""
    betas = np.asarray(betas0, np.float64).copy()
    history = []
    for it in range(iterations):
        n = len(instances)
        ctx = create_instances(instances, [betas] * n, Config(update=update, seed=seed + it),
                               instance_ids=list(range(n)), stream=stream)
        run_cycles(ctx, sweeps)
        acc = np.zeros(len(betas) - 1, np.int64)
        att = np.zeros(len(betas) - 1, np.int64)
        for k in range(n):
            sa, st, _, _ = read_stats(ctx, k)
            acc += sa
            att += st
        destroy(ctx)
        history.append({"betas": betas.copy(), "acceptance": acc / np.maximum(att, 1)})
        betas = respace(betas, pair_distance(acc, att))
    return betas, history
