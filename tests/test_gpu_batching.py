"""Batching machinery of the C ABI: concurrent size-class groups, the block-size autotuner,
CUDA-graph replay of the fused cycle, and slot replacement / activation for continuous
batching. Every check compares exact integer results (spins, energies, walker labels)."""
import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2509_23043_gb300 as pt

pytestmark = pytest.mark.gpu


def _state(ctx, k):
    s, E = pt.read_state(ctx, k)
    return s, E, pt.read_walkers(ctx, k), pt.read_counters(ctx, k)[0]


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _ragged(P=8):
    Ls = [6, 8, 7, 10, 6, 12]
    Rs = [24, 40, 16, 32, 24, 48]
    insts = [I.ea_instance(L, index=300 + k) for k, L in enumerate(Ls)]
    betas = [I.geometric_betas(0.1, 3.0, R) for R in Rs]
    props = [[1] * (R - 2) + [0, 0] for R in Rs]
    ids = [7000 + k for k in range(len(Ls))]
    pools = [[I.random_configs(insts[k].n_spins, P, seed=5, index=100 * k + r) for r in range(Rs[k])]
             for k in range(len(Ls))]
    return insts, betas, props, ids, pools


def _make(cfg, data):
    insts, betas, props, ids, pools = data
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=props, instance_ids=ids)
    for k in range(len(insts)):
        for r in range(len(betas[k])):
            pt.load_proposals(ctx, k, r, pools[k][r])
    return ctx


def test_groups_run_concurrently_and_match_oracle():
    data = _ragged()
    cfg = pt.Config(seed=11, propose_every=3, pool_size=8)
    ctx = _make(cfg, data)
    groups = pt.group_info(ctx)
    assert len(groups) == 5 and sum(g["members"] for g in groups) == 6   # (L, W) classes
    pt.run_cycles(ctx, 17)
    insts, betas, props, ids, pools = data
    for k in (0, 2, 5):
        o = O.Oracle(insts[k], betas[k], instance_id=ids[k], prop_enabled=props[k],
                     propose_every=3, seed=11, pool_size=8)
        for r in range(len(betas[k])):
            o.load_pool(r, pools[k][r])
        o.run_cycles(17)
        s, E, w = o.read()
        g = _state(ctx, k)
        assert np.array_equal(g[0], s) and np.array_equal(g[1], E) and np.array_equal(g[2], w)


@pytest.mark.parametrize("update", [0, 1])
def test_autotune_leaves_the_run_unchanged(update):
    data = _ragged()
    cfg = pt.Config(seed=12, propose_every=2, pool_size=8, update=update)
    a, b = _make(cfg, data), _make(cfg, data)
    pt.run_cycles(a, 5)
    pt.run_cycles(b, 5)
    chosen = pt.autotune(b, probe_cycles=4)
    assert len(chosen) == len(pt.group_info(b)) and all(t % 32 == 0 for t in chosen)
    pt.run_cycles(a, 9)
    pt.run_cycles(b, 9)
    for k in range(6):
        _same(_state(a, k), _state(b, k))


@pytest.mark.parametrize("update", [0, 1])
def test_graph_replay_equals_direct_launches(update):
    data = _ragged()
    cfg = pt.Config(seed=13, propose_every=2, pool_size=8, update=update)
    a, b = _make(cfg, data), _make(cfg, data)
    pt.run_cycles(a, 30)
    for _ in range(3):
        pt.run_cycles_graph(b, 10)
    for k in range(6):
        _same(_state(a, k), _state(b, k))


@pytest.mark.parametrize("update", [0, 1])
def test_slot_replacement_and_deactivation(update):
    R = 16
    betas = I.geometric_betas(0.2, 3.0, R)
    insts = [I.ea_instance(6, index=k) for k in range(3)]
    cfg = pt.Config(seed=14, update=update)
    ctx = pt.create_instances(insts, [betas] * 3, cfg, instance_ids=[1, 2, 3])
    pt.run_cycles(ctx, 8)
    frozen = _state(ctx, 1)
    pt.set_active(ctx, 1, False)
    pt.run_cycles(ctx, 8)
    _same(frozen, _state(ctx, 1))                    # an inactive slot does not move
    new = I.ea_instance(6, index=77)
    pt.set_instance(ctx, 1, new, betas, instance_id=99)
    pt.run_cycles(ctx, 12)
    alone = pt.create_instances([new], [betas], cfg, instance_ids=[99])
    pt.run_cycles(alone, 12)
    _same(_state(alone, 0), _state(ctx, 1))          # same result alone and in the mix
    with pytest.raises(pt.PTError):
        pt.set_instance(ctx, 1, I.ea_instance(8, index=1), betas, instance_id=5)
