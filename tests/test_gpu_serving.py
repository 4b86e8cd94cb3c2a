"""The continuous-batching server: requests of different sizes arrive while others run,
share launches, and retire at their target. Each request's result (sweeps to target, best
energy, final configuration) is the same in the mix as alone, and the reported energies are
those of the configurations (checked with the oracle)."""
import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2509_23043_gb300 as pt
from paper_2509_23043_gb300 import serve as S

pytestmark = pytest.mark.gpu


def _requests():
    R, P = 16, 32
    betas = I.geometric_betas(0.1, 3.0, R)
    prop = [1] * (R - 2) + [0, 0]
    Ls = [6, 8, 6, 8, 7, 6]
    insts = [I.ea_instance(L, index=500 + k) for k, L in enumerate(Ls)]
    ids = [4000 + k for k in range(len(Ls))]
    pools = S.make_pools(insts, [betas] * len(Ls), ids, P, burnin=300, gap=2)
    eref = S.reference_energies(insts, [betas] * len(Ls), ids, sweeps=4000)
    reqs = [S.Request(ids[k], insts[k], betas, prop, pools[k], eref[k], arrival=0.002 * k)
            for k in range(len(Ls))]
    return reqs, betas, prop, P


def test_served_results_equal_alone_results():
    # Requests that arrive while others run share launches with them, yet each one's whole
    # trajectory is its own: the sweeps to the target, the best energy, and the final spins,
    # energies and walker labels of every slot are the same in the mix as alone.
    reqs, betas, prop, P = _requests()
    cfg = pt.Config(seed=77, propose_every=10, pool_size=P)
    srv = S.TaptServer({6: 2, 7: 1, 8: 1}, betas, prop, cfg, tick_cycles=20, keep_final=True)
    done = srv.serve(reqs, budget_sweeps=4000)
    assert len(done) == len(reqs)
    for r in done:
        alone = S.Request(r.rid, r.instance, r.betas, r.prop, r.pool, r.e_ref)
        S.run_alone(alone, cfg, budget_sweeps=4000, tick_cycles=20, keep_final=True)
        assert alone.sweeps == r.sweeps and alone.best == r.best
        for mixed, own in zip(r.final, alone.final):     # spins, energies, walker labels
            assert np.array_equal(mixed, own)
        for k in range(len(betas)):                      # the energies are the states'
            assert r.final[1][k] == O.energy(r.instance, r.final[0][k])
    summary = S.summarize(done)
    assert summary["requests"] == len(reqs)


def test_reported_energy_is_the_configuration_energy():
    reqs, betas, prop, P = _requests()
    r = reqs[1]
    cfg = pt.Config(seed=78, propose_every=10, pool_size=P)
    ctx = pt.create_instances([r.instance], [betas], cfg, prop_enabled=[prop], instance_ids=[r.rid])
    pt.load_proposals_inst_packed(ctx, 0, r.pool)
    pt.run_cycles(ctx, 300)
    s, E = pt.read_state(ctx, 0)
    for k in range(len(betas)):
        assert E[k] == O.energy(r.instance, s[k])
    # the pool entries round-trip: entry 3 of slot 2 decodes to a +-1 configuration whose
    # energy the oracle evaluates like any other
    cfgs = I.unpack_bits(r.pool[3], r.instance.n_spins)
    assert cfgs.shape == (len(betas), r.instance.n_spins)
    assert isinstance(O.energy(r.instance, cfgs[2]), int)
