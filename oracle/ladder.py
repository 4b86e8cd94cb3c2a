"""Oracle of the ladder optimisation (test infrastructure only; written independently of the
library's version): PT runs by the C oracle, then the re-spacing written out with plain
loops. The distance of a pair is d = 2 erfcinv(A), A clipped to [1e-4, 1 - 1e-9]. The new
point k lies where the cumulative distance, linear between old points, reaches k/(R-1) of
the total. erfcinv is found by bisection on math.erfc."""
from __future__ import annotations

import math

from . import Oracle


def erfcinv(y: float) -> float:
    lo, hi = -6.0, 6.0            # erfc is decreasing: erfc(-6) ~ 2, erfc(6) ~ 2e-17
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.erfc(mid) > y:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def distances(acc, att):
    out = []
    for a, t in zip(acc, att):
        A = a / max(t, 1)
        A = min(max(A, 1e-4), 1.0 - 1e-9)
        out.append(2.0 * erfcinv(A))
    return out


def respace(betas, d):
    R = len(betas)
    cum = [0.0]
    for x in d:
        cum.append(cum[-1] + x)
    new = [betas[0]]
    for k in range(1, R - 1):
        target = cum[-1] * k / (R - 1)
        j = 0
        while j < R - 2 and cum[j + 1] < target:
            j += 1
        span = cum[j + 1] - cum[j]
        f = 0.0 if span <= 0 else (target - cum[j]) / span
        new.append(betas[j] + f * (betas[j + 1] - betas[j]))
    new.append(betas[-1])
    return new


def optimise_ladder(instances, betas0, iterations=5, sweeps=2000, update=0, seed=0x1ADD):
    betas = [float(b) for b in betas0]
    history = []
    for it in range(iterations):
        acc = [0] * (len(betas) - 1)
        att = [0] * (len(betas) - 1)
        for k, inst in enumerate(instances):
            o = Oracle(inst, betas, instance_id=k, update=update, seed=seed + it)
            o.run_cycles(sweeps)
            sa, st, _, _ = o.stats()
            for r in range(len(acc)):
                acc[r] += int(sa[r])
                att[r] += int(st[r])
        history.append({"betas": list(betas), "accepted": acc, "attempted": att})
        betas = respace(betas, distances(acc, att))
    return betas, history
