"""The proposal rules on the GPU: parity of the always-accept rule with the oracle, and the
transition-matrix result of Supplementary S2 (Fig. S2) reproduced at scale.

The large test runs 2048 independent copies of the three-replica full-adder system of
Supplementary S2 (beta = {0.5, 1.7, 4.6}, proposals from exact Boltzmann draws on the two
hottest slots, Gibbs sweeps). It compares each slot's long-run energy histogram with the
exact chain's stationary law, built in tests/test_transition_matrix.py from the definitions
of the sweep, swap and proposal matrices. Under the Delta-E-only rule the proposal-receiving
slots follow the exact biased law, not the Boltzmann law. Under always-accept every slot
follows the Boltzmann law."""
import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2509_23043_gb300 as pt
from test_transition_matrix import BETAS, LAWS, _energy, _fa, _pi, _q_product, _states, _stationary

pytestmark = pytest.mark.gpu


def _same(ctx, k, o):
    s, E = pt.read_state(ctx, k)
    so, Eo, wo = o.read()
    assert np.array_equal(E, Eo)
    assert np.array_equal(pt.read_walkers(ctx, k), wo)
    assert np.array_equal(s, so)


@pytest.mark.parametrize("engine", ["lattice", "graph"])
def test_always_accept_rule_matches_oracle(engine):
    if engine == "lattice":
        inst, R, update = I.ea_instance(6, index=12), 12, 0
    else:
        inst, R, update = I.multiplier(3).instance(35), 10, 1
    P = 6
    betas = I.geometric_betas(0.1, 3.0, R)
    prop = [1] * (R - 2) + [0, 0]
    cfg = pt.Config(update=update, seed=0x51, propose_every=3, propose_start=0, pool_size=P,
                    proposal_rule=pt.ALWAYS_ACCEPT)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[21])
    assert pt.info(ctx)["engine"] == engine
    o = O.Oracle(inst, betas, instance_id=21, prop_enabled=prop, update=update,
                 propose_every=3, seed=0x51, pool_size=P, proposal_rule=1)
    for r in range(R):
        pool = I.random_configs(inst.n_spins, P, seed=77, index=r)
        pt.load_proposals(ctx, 0, r, pool)
        o.load_pool(r, pool)
    for chunk in (2, 9, 20):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _same(ctx, 0, o)
    _, _, pa, ptot = pt.read_stats(ctx, 0)
    assert np.array_equal(pa, ptot) and ptot[0] > 0


def test_rule_out_of_range_rejected():
    with pytest.raises(pt.PTError):
        pt.create_instances([I.ea_instance(4)], [[0.5, 1.0]], pt.Config(proposal_rule=3))
    with pytest.raises(pt.PTError):          # the MH rule needs pool proposals
        pt.create_instances([I.ea_instance(4)], [[0.5, 1.0]],
                            pt.Config(proposal_rule=2, proposal_source=1))


@pytest.mark.parametrize("engine,R", [("lattice", 12), ("lattice", 40), ("graph", 10), ("graph", 36)])
def test_independent_mh_rule_matches_oracle(engine, R):
    # proposal_rule 2 (Supplementary S2, the MH rule) with product-Bernoulli laws loaded per
    # slot (some slots left at the uniform law): spins, energies, walkers, decisions and
    # statistics bit-exact against the oracle, after several chunk sizes
    if engine == "lattice":
        inst, update = I.ea_instance(6, index=13), 0
    else:
        inst, update = I.multiplier(3).instance(35), 1
    P = 8
    N = inst.n_spins
    betas = I.geometric_betas(0.002, 0.5, R)     # hot: random entries are sometimes accepted
    prop = [1] * (R - 2) + [0, 0]
    cfg = pt.Config(update=update, seed=0x52, propose_every=2, propose_start=0, pool_size=P,
                    proposal_rule=pt.INDEPENDENT_MH)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[22])
    assert pt.info(ctx)["engine"] == engine
    o = O.Oracle(inst, betas, instance_id=22, prop_enabled=prop, update=update,
                 propose_every=2, seed=0x52, pool_size=P, proposal_rule=2)
    g = np.random.default_rng(31)
    for r in range(R):
        law = g.uniform(0.45, 0.55, size=N)
        pool = np.where(g.random((P, N)) < law[None, :], 1, -1).astype(np.int8)
        pt.load_proposals(ctx, 0, r, pool)
        o.load_pool(r, pool)
        if r % 5 != 4:                        # every fifth slot keeps the uniform law
            pt.load_proposal_law(ctx, 0, r, law)
            o.load_law(r, law)
    for chunk in (2, 7, 21):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _same(ctx, 0, o)
    sa, st, pa, ptot = pt.read_stats(ctx, 0)
    osa, ost, opa, optot = o.stats()
    assert np.array_equal(pa, opa) and np.array_equal(ptot, optot)
    assert 0 < pa.sum() < ptot.sum()          # some proposals accepted, some rejected


def test_proposal_law_needs_the_mh_rule():
    ctx = pt.create_instances([I.ea_instance(4)], [[0.5, 1.0]], pt.Config(pool_size=2))
    with pytest.raises(pt.PTError) as e:
        pt.load_proposal_law(ctx, 0, 0, np.full(64, 0.5))
    assert e.value.status == pt.PT_ESTATE
    ctx2 = pt.create_instances([I.ea_instance(4)], [[0.5, 1.0]],
                               pt.Config(pool_size=2, proposal_rule=pt.INDEPENDENT_MH))
    with pytest.raises(pt.PTError):
        pt.load_proposal_law(ctx2, 0, 0, np.full(64, 1.0))   # outside (0, 1)


def _energy_marginals(p_states, E):
    levels = np.unique(E)
    return levels, np.array([p_states[E == e].sum() for e in levels])


@pytest.mark.parametrize("rule", [pt.DELTA_E_ONLY, pt.ALWAYS_ACCEPT])
def test_full_adder_chain_at_scale_follows_the_exact_stationary_law(rule):
    inst = _fa()
    S = _states()
    E = _energy(inst, S)
    exact, pis, _ = _stationary("delta_e" if rule == pt.DELTA_E_ONLY else "always")
    n, P = 2048, 1024                               # 1000 events: no entry is reused
    g = np.random.default_rng(99 + rule)
    cfg = pt.Config(update=pt.GIBBS, seed=0xF52, propose_every=1, propose_start=0, pool_size=P,
                    proposal_rule=rule)
    ctx = pt.create_instances([inst] * n, [BETAS] * n, cfg, prop_enabled=[[1, 1, 0]] * n,
                              instance_ids=list(range(n)))
    # entry-major pools: [entry][instance][slot][1 word], exact Boltzmann draws for slots 0, 1
    words = np.zeros((P, n, 3), dtype=np.uint32)
    bits = (S > 0).astype(np.uint32) @ (1 << np.arange(5)).astype(np.uint32)
    for r in range(2):
        words[:, :, r] = bits[g.choice(32, size=(P, n), p=_pi(E, BETAS[r]))]
    pt.load_proposals_packed(ctx, words.reshape(P, -1), 0, P)
    pt.run_cycles(ctx, 400)
    levels = np.unique(E)
    counts = np.zeros((3, len(levels)))
    steps = 600
    for _ in range(steps):
        pt.run_cycles(ctx, 1)
        Es = np.stack(pt.energies(ctx))             # [n][3], slot order
        for r in range(3):
            counts[r] += (Es[:, r][:, None] == levels[None, :]).sum(0)
    total = n * steps
    for r in range(3):
        q = counts[r] / total
        _, m = _energy_marginals(exact[r], E)
        _, b = _energy_marginals(pis[r], E)
        # successive cycles are correlated: allow for an effective sample 50x smaller
        noise = 0.5 * np.sum(np.sqrt(m * (1 - m) / (total / 50)))
        assert 0.5 * np.abs(q - m).sum() < 4 * noise + 1e-3, (rule, r, q, m)
        if rule == pt.DELTA_E_ONLY and r < 2:
            # biased, as Fig. S2 shows: the exact energy-law distance is 0.16 (slot 0) and
            # 0.041 (slot 1); at the cold slot it is 8e-5, below this test's resolution
            assert 0.5 * np.abs(q - b).sum() > 4 * noise + 1e-3


def test_full_adder_mh_rule_at_scale_keeps_boltzmann():
    # proposal_rule 2 on 2048 copies of the S2 system, the two hottest slots proposed from
    # pools drawn from product-Bernoulli laws far from their Boltzmann laws (the laws loaded
    # beside them): every slot's energy law is the Boltzmann law, as the exact MH chain's.
    # (The Delta-E-only rule with the same pools is biased at the level of states, KL > 1e-3
    # in tests/test_transition_matrix.py, but its energy laws stay within 0.01 of Boltzmann,
    # below this test's resolution.)
    inst = _fa()
    S = _states()
    E = _energy(inst, S)
    exact, pis, _ = _stationary("mh")
    n, P = 2048, 1024
    g = np.random.default_rng(103)
    cfg = pt.Config(update=pt.GIBBS, seed=0xF53, propose_every=1, propose_start=0, pool_size=P,
                    proposal_rule=pt.INDEPENDENT_MH)
    ctx = pt.create_instances([inst] * n, [BETAS] * n, cfg, prop_enabled=[[1, 1, 0]] * n,
                              instance_ids=list(range(n)))
    words = np.zeros((P, n, 3), dtype=np.uint32)
    bits = (S > 0).astype(np.uint32) @ (1 << np.arange(5)).astype(np.uint32)
    for r in range(2):
        words[:, :, r] = bits[g.choice(32, size=(P, n), p=_q_product(LAWS[r]))]
    pt.load_proposals_packed(ctx, words.reshape(P, -1), 0, P)
    for k in range(n):
        for r in range(2):
            pt.load_proposal_law(ctx, k, r, LAWS[r])
    pt.run_cycles(ctx, 400)
    levels = np.unique(E)
    counts = np.zeros((3, len(levels)))
    steps = 600
    for _ in range(steps):
        pt.run_cycles(ctx, 1)
        Es = np.stack(pt.energies(ctx))
        for r in range(3):
            counts[r] += (Es[:, r][:, None] == levels[None, :]).sum(0)
    total = n * steps
    for r in range(3):
        q = counts[r] / total
        _, m = _energy_marginals(exact[r], E)
        _, b = _energy_marginals(pis[r], E)
        assert np.allclose(m, b, atol=1e-9)             # the exact MH chain is Boltzmann
        noise = 0.5 * np.sum(np.sqrt(m * (1 - m) / (total / 50)))
        assert 0.5 * np.abs(q - m).sum() < 4 * noise + 1e-3, (r, q, m)
