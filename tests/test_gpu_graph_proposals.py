"""Global proposals on the graph engine against the oracle (Eq. 2): every enabled slot's
entry, clamps applied, its exact energy, the decision and the copy. Covers more than 32 slots
(two slot groups), duplicate edges, couplings of several values and signs, sites without a
field, graphs without edges or without fields, couplings too large for the packed rows,
both local rules and both proposal rules. Compared bit for bit: spins, energies, walker
labels and acceptance statistics."""
import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2509_23043_gb300 as pt

pytestmark = pytest.mark.gpu


def _random_graph(n, n_edges, jmax, hmax, seed, clamp_frac=0.1, dup=0):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, size=n_edges)
    b = (a + rng.integers(1, n, size=n_edges)) % n            # never a self loop
    J = rng.integers(1, jmax + 1, size=n_edges) * rng.choice([-1, 1], size=n_edges)
    if dup:                                                   # repeat some edges verbatim
        k = rng.integers(0, n_edges, size=dup)
        a, b, J = np.concatenate([a, a[k]]), np.concatenate([b, b[k]]), np.concatenate([J, J[k]])
    h = None if hmax == 0 else rng.integers(-hmax, hmax + 1, size=n).astype(np.int32)
    cl = np.zeros(n, np.int8)
    m = rng.random(n) < clamp_frac
    cl[m] = rng.choice([-1, 1], size=int(m.sum())).astype(np.int8)
    return I.Instance(n, a.astype(np.int32), b.astype(np.int32), J.astype(np.int32), h, cl, 0)


def _same(ctx, k, o):
    s, E = pt.read_state(ctx, k)
    so, Eo, wo = o.read()
    assert np.array_equal(E, Eo)
    assert np.array_equal(pt.read_walkers(ctx, k), wo)
    assert np.array_equal(s, so)
    for x, y in zip(pt.read_stats(ctx, k), o.stats()):
        assert np.array_equal(x, y)


CASES = {
    "R40_dup": dict(n=77, n_edges=160, jmax=5, hmax=3, R=40, n_prop=35, dup=12, b0=0.02),
    "R33_nofield": dict(n=64, n_edges=120, jmax=3, hmax=0, R=33, n_prop=33, dup=0, b0=0.02),
    "R12_largeJ": dict(n=45, n_edges=90, jmax=60, hmax=20, R=12, n_prop=9, dup=4, b0=0.0005),
    "R70_sparse": dict(n=31, n_edges=20, jmax=2, hmax=1, R=70, n_prop=64, dup=0, b0=0.02),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("update,rule", [(1, 0), (0, 0), (1, 1)])
def test_graph_proposals_match_oracle(case, update, rule):
    c = CASES[case]
    inst = _random_graph(c["n"], c["n_edges"], c["jmax"], c["hmax"], seed=len(case) * 7 + update,
                         dup=c["dup"])
    R, P = c["R"], 6
    betas = I.geometric_betas(c["b0"], 3.0, R)
    prop = [1] * c["n_prop"] + [0] * (R - c["n_prop"])
    cfg = pt.Config(update=update, seed=0x6A, propose_every=2, propose_start=1, pool_size=P,
                    proposal_rule=rule)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[77])
    assert pt.info(ctx)["engine"] == "graph"
    o = O.Oracle(inst, betas, instance_id=77, prop_enabled=prop, update=update,
                 propose_every=2, propose_start=1, seed=0x6A, pool_size=P, proposal_rule=rule)
    for r in range(R):
        pool = I.random_configs(inst.n_spins, P, seed=0x6B, index=r)
        pt.load_proposals(ctx, 0, r, pool)
        o.load_pool(r, pool)
    for chunk in (2, 5, 24):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _same(ctx, 0, o)
    _, _, pa, ptot = pt.read_stats(ctx, 0)
    assert ptot.sum() > 0 and pa.sum() > 0
    if rule == 1:
        assert np.array_equal(pa, ptot)


def test_graph_proposals_without_edges_and_through_the_manual_api():
    insts = [_random_graph(40, 0, 1, 4, seed=3), _random_graph(50, 100, 4, 2, seed=4)]
    Rs = [8, 36]
    betas = [I.geometric_betas(0.05, 2.0, R) for R in Rs]
    props = [[1] * R for R in Rs]
    P = 4
    cfg = pt.Config(update=1, seed=0x6C, propose_every=3, pool_size=P)
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=props, instance_ids=[5, 6])
    os_ = [O.Oracle(insts[k], betas[k], instance_id=5 + k, prop_enabled=props[k], update=1,
                    propose_every=3, seed=0x6C, pool_size=P) for k in range(2)]
    for k in range(2):
        for r in range(Rs[k]):
            pool = I.random_configs(insts[k].n_spins, P, seed=0x6D + k, index=r)
            pt.load_proposals(ctx, k, r, pool)
            os_[k].load_pool(r, pool)
    pt.run_cycles(ctx, 7)
    for o in os_:
        o.run_cycles(7)
    for _ in range(3):
        pt.sweep(ctx, 1)
        pt.global_propose(ctx)
        pt.exchange(ctx)
        for o in os_:
            o.sweeps(1)
            o.propose()
            o.exchange()
    for k, o in enumerate(os_):
        _same(ctx, k, o)
