"""Parity at the full sizes of the benchmark configurations, in the launch configuration the
benchmark uses (automatic block shapes, groups, autotuner and graph replay where it uses
them): sampled instances are rerun by the oracle one by one and must agree exactly; every
instance must satisfy properties that hold at any size (energy of the configuration, walker
labels form a permutation, clamped spins untouched)."""
import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2509_23043_gb300 as pt

pytestmark = pytest.mark.gpu


def _energy_all(inst, spins):
    """Energies of a batch of configurations [k][N] (vectorised, for the property checks)."""
    s = spins.astype(np.int64)
    E = -(inst.edge_J[None, :] * s[:, inst.edge_i] * s[:, inst.edge_j]).sum(1)
    if inst.h is not None:
        E -= (inst.h[None, :] * s).sum(1)
    return E


def _check_properties(ctx, insts, which=None):
    for k in (range(len(insts)) if which is None else which):
        inst = insts[k]
        s, E = pt.read_state(ctx, k)
        assert np.array_equal(_energy_all(inst, s), E.astype(np.int64)), f"instance {k}"
        w = pt.read_walkers(ctx, k)
        assert sorted(w.tolist()) == list(range(len(E)))
        if inst.clamp is not None:
            cl = inst.clamp != 0
            assert np.all(s[:, cl] == inst.clamp[cl][None, :])


def _compare(ctx, k, o):
    s, E = pt.read_state(ctx, k)
    so, Eo, wo = o.read()
    assert np.array_equal(E, Eo) and np.array_equal(pt.read_walkers(ctx, k), wo)
    assert np.array_equal(s, so)


def test_config1_plain_pt_full_run():
    # one EA instance, L=6, 16 replicas, beta 0.2 -> 3.0, 10^4 sweeps, no proposals
    inst = I.ea_instance(6, index=0)
    betas = I.geometric_betas(0.2, 3.0, 16)
    cfg = pt.Config(seed=0x7A972509)
    ctx = pt.create_instances([inst], [betas], cfg, instance_ids=[0])
    pt.run_cycles(ctx, 10_000)
    o = O.Oracle(inst, betas, instance_id=0, seed=0x7A972509)
    o.run_cycles(10_000)
    _compare(ctx, 0, o)
    c, _ = pt.read_counters(ctx, 0)
    assert list(c) == [10_000, 10_000, 0]


@pytest.mark.parametrize("update", [pt.METROPOLIS, pt.GIBBS])
def test_config2_batched_tapt_sampled(update):
    # 256 EA L=10, R=32, pools of 1024 per slot, proposals every 10 sweeps from sweep 100 on
    # the 30 hottest slots (the benchmark's layout and launch shape), Metropolis (the
    # benchmark's rule) and Gibbs
    B, R, P = 256, 32, 1024
    insts = [I.ea_instance(10, index=k) for k in range(B)]
    betas = [I.geometric_betas(0.1, 3.0, R)] * B
    prop = [[1] * (R - 2) + [0, 0]] * B
    cfg = pt.Config(seed=0x7A972509, propose_every=10, propose_start=100, pool_size=P,
                    update=update)
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=prop, instance_ids=list(range(B)))
    assert pt.info(ctx)["threads"] == 256
    samples = (0, 131, 255)
    pools = {k: [I.random_configs(1000, P, seed=9, index=100 * k + r) for r in range(R)]
             for k in samples}
    for k in samples:
        for r in range(R):
            pt.load_proposals(ctx, k, r, pools[k][r])
    pt.run_cycles(ctx, 130)
    for k in samples:
        o = O.Oracle(insts[k], betas[k], instance_id=k, prop_enabled=prop[k], propose_every=10,
                     propose_start=100, seed=0x7A972509, pool_size=P, update=update)
        for r in range(R):
            o.load_pool(r, pools[k][r])
        o.run_cycles(130)
        assert o.counters()[2] > 0
        _compare(ctx, k, o)
    _check_properties(ctx, insts)


def test_config3_ragged_persistent_sampled():
    # 4096 EA instances, L uniform in {6..16} (even), R uniform in 24..48, proposals every
    # 10 from pools of 512, autotuned block sizes, graph-replayed cycles
    g = np.random.default_rng(3)
    n, P = 4096, 512
    Ls = g.choice([6, 8, 10, 12, 14, 16], size=n)
    Rs = g.integers(24, 49, size=n)
    insts = [I.ea_instance(int(L), index=k) for k, L in enumerate(Ls)]
    betas = [I.geometric_betas(0.1, 3.0, int(R)) for R in Rs]
    props = [[1] * (int(R) - 2) + [0, 0] for R in Rs]
    cfg = pt.Config(seed=0x7A972509, propose_every=10, propose_start=0, pool_size=P)
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=props, instance_ids=list(range(n)))
    assert len(pt.group_info(ctx)) > 6
    samples = [int(np.argmin(Ls * 100 + Rs)), int(np.argmax(Ls * 100 + Rs)), 1000, 4095]
    pools = {k: [I.random_configs(int(Ls[k]) ** 3, P, seed=11, index=100 * k + r)
                 for r in range(int(Rs[k]))] for k in samples}
    for k in samples:
        for r in range(int(Rs[k])):
            pt.load_proposals(ctx, k, r, pools[k][r])
    pt.autotune(ctx, probe_cycles=4)
    for _ in range(2):
        pt.run_cycles_graph(ctx, 10)
    for k in samples:
        o = O.Oracle(insts[k], betas[k], instance_id=k, prop_enabled=props[k], propose_every=10,
                     seed=0x7A972509, pool_size=P)
        for r in range(int(Rs[k])):
            o.load_pool(r, pools[k][r])
        o.run_cycles(20)
        _compare(ctx, k, o)
    for k in range(0, n, 97):      # property checks on a spread of the batch
        s, E = pt.read_state(ctx, k)
        assert np.array_equal(_energy_all(insts[k], s), E.astype(np.int64))


@pytest.mark.parametrize("update,every", [(pt.GIBBS, 10), (pt.METROPOLIS, 10), (pt.GIBBS, 1)])
def test_config4_factorization_sampled(update, every):
    # 1000 products of two primes <= 255 on the 8x8-bit multiplier (N=200), product bits and
    # carry-ins clamped, R=32, beta 0.05 -> 5.0, Gibbs or Metropolis, pool proposals every 10
    # sweeps (the factorization workload) or every sweep (the time-to-solution workload)
    mult = I.multiplier(8)
    prods = I.draw_prime_products(1000)
    insts = [mult.instance(C) for C, _, _ in prods]
    R, P = 32, 16
    betas = [I.geometric_betas(0.05, 5.0, R)] * len(insts)
    prop = [[1] * 23 + [0] * 9] * len(insts)
    cfg = pt.Config(update=update, seed=0x7A972509, propose_every=every, propose_start=0,
                    pool_size=P)
    ids = list(range(len(insts)))
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=prop, instance_ids=ids)
    assert pt.info(ctx)["engine"] == "graph"
    samples = (0, 499, 999)
    pools = {k: [I.random_configs(200, P, seed=13, index=100 * k + r) for r in range(R)]
             for k in samples}
    for k in samples:
        for r in range(R):
            pt.load_proposals(ctx, k, r, pools[k][r])
    pt.run_cycles(ctx, 40)
    for k in samples:
        o = O.Oracle(insts[k], betas[k], instance_id=k, prop_enabled=prop[k], update=update,
                     propose_every=every, seed=0x7A972509, pool_size=P)
        for r in range(R):
            o.load_pool(r, pools[k][r])
        o.run_cycles(40)
        _compare(ctx, k, o)
    _check_properties(ctx, insts, range(0, len(insts), 50))


@pytest.mark.parametrize("update", [0, 1])
def test_maximal_walker_blocks_and_single_replica(update):
    inst = I.ea_instance(16, index=4)
    for R in (128, 1):
        betas = I.geometric_betas(0.3, 2.0, R)
        ctx = pt.create_instances([inst], [betas], pt.Config(seed=5, update=update),
                                  instance_ids=[3])
        pt.run_cycles(ctx, 3)
        o = O.Oracle(inst, betas, instance_id=3, seed=5, update=update)
        o.run_cycles(3)
        _compare(ctx, 0, o)
