"""Contextual proposals (Supplementary S3) on the GPU against the oracle: every enabled slot
keeps a random 2^-k of its sites and refills the rest by Metropolis sweeps at its beta; the
result is accepted by the proposal rule. Compared bit for bit: spins, energies, walker
labels, counters and acceptance statistics."""
import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2509_23043_gb300 as pt

pytestmark = pytest.mark.gpu


def _same(ctx, k, o):
    s, E = pt.read_state(ctx, k)
    so, Eo, wo = o.read()
    assert np.array_equal(E, Eo)
    assert np.array_equal(pt.read_walkers(ctx, k), wo)
    assert np.array_equal(s, so)
    g = pt.read_stats(ctx, k)
    for a, b in zip(g, o.stats()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("L,R,n_prop,log2,sweeps,rule", [
    (4, 12, 10, 1, 1, 0), (4, 12, 10, 2, 3, 1), (5, 9, 7, 3, 2, 0), (6, 40, 30, 1, 2, 0),
    (3, 33, 32, 2, 1, 0)])
def test_contextual_proposals_match_oracle(L, R, n_prop, log2, sweeps, rule):
    inst = I.ea_instance(L, index=50 + L + R)
    betas = I.geometric_betas(0.1, 3.0, R)
    prop = [1] * n_prop + [0] * (R - n_prop)
    cfg = pt.Config(seed=0xC7, propose_every=3, propose_start=0, proposal_rule=rule,
                    proposal_source=pt.CONTEXT, context_log2=log2, context_sweeps=sweeps)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[31])
    assert pt.info(ctx)["engine"] == "lattice"
    o = O.Oracle(inst, betas, instance_id=31, prop_enabled=prop, propose_every=3, seed=0xC7,
                 proposal_rule=rule, proposal_source=1, context_log2=log2,
                 context_sweeps=sweeps)
    _same(ctx, 0, o)
    for chunk in (3, 10, 17):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _same(ctx, 0, o)
    _, _, pa, ptot = pt.read_stats(ctx, 0)
    assert ptot[0] == 10 and pa.sum() > 0
    if rule == 1:
        assert np.array_equal(pa, ptot)


def test_contextual_proposals_in_a_batch_and_through_the_manual_api():
    insts = [I.ea_instance(4, index=k) for k in range(3)] + [I.ea_instance(6, index=9)]
    Rs = [8, 8, 20, 16]
    betas = [I.geometric_betas(0.2, 2.5, R) for R in Rs]
    props = [[1] * (R - 1) + [0] for R in Rs]
    cfg = pt.Config(seed=0xC8, propose_every=2, proposal_source=pt.CONTEXT, context_log2=2,
                    context_sweeps=2)
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=props, instance_ids=[5, 6, 7, 8])
    os_ = [O.Oracle(insts[k], betas[k], instance_id=5 + k, prop_enabled=props[k],
                    propose_every=2, seed=0xC8, proposal_source=1, context_log2=2,
                    context_sweeps=2) for k in range(4)]
    pt.run_cycles(ctx, 9)
    for o in os_:
        o.run_cycles(9)
    pt.sweep(ctx, 2)
    pt.global_propose(ctx)
    pt.exchange(ctx)
    for o in os_:
        o.sweeps(2)
        o.propose()
        o.exchange()
    for k, o in enumerate(os_):
        _same(ctx, k, o)


def test_contextual_proposals_rejected_where_unsupported():
    mult = I.multiplier(2).instance(6)
    with pytest.raises(pt.PTError):          # graph engine
        pt.create_instances([mult], [[0.5, 1.0]], pt.Config(proposal_source=pt.CONTEXT))
    inst = I.ea_instance(4)
    with pytest.raises(pt.PTError):          # more than 32 enabled slots
        pt.create_instances([inst], [I.geometric_betas(0.1, 2.0, 40)],
                            pt.Config(proposal_source=pt.CONTEXT), prop_enabled=[[1] * 40])
    with pytest.raises(pt.PTError):          # kept fraction 2^-4
        pt.create_instances([inst], [[0.5, 1.0]],
                            pt.Config(proposal_source=pt.CONTEXT, context_log2=4))
    with pytest.raises(pt.PTError):          # Gibbs sweeps (the refill is Metropolis)
        pt.create_instances([inst], [[0.5, 1.0]],
                            pt.Config(update=pt.GIBBS, proposal_source=pt.CONTEXT))
