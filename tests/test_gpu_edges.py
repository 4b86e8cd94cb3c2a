"""Edge cases of the GPU path against the oracle: the largest lattice the engine takes, graphs
with no edges or with every spin clamped, a single-site graph, zero-length calls, an empty
batch, and proposals with a pool of one entry."""
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


@pytest.mark.parametrize("update", [0, 1])
def test_largest_lattice_L20_R32(update):
    inst = I.ea_instance(20, index=2)                  # N = 8000, the engine's limit
    betas = I.geometric_betas(0.2, 2.5, 32)
    ctx = pt.create_instances([inst], [betas], pt.Config(seed=9, update=update), instance_ids=[4])
    assert pt.info(ctx)["engine"] == "lattice"
    pt.run_cycles(ctx, 4)
    o = O.Oracle(inst, betas, instance_id=4, seed=9, update=update)
    o.run_cycles(4)
    _same(ctx, 0, o)


def test_lattice_beyond_limits_rejected():
    with pytest.raises(pt.PTError):                    # N > 8192
        pt.create_instances([I.ea_instance(21)], [I.geometric_betas(0.2, 2.0, 4)], pt.Config())
    # too large for shared memory: accepted, spins and table in global memory ...
    ctx = pt.create_instances([I.ea_instance(20)], [I.geometric_betas(0.2, 2.0, 64)], pt.Config())
    assert pt.group_info(ctx)[0]["smem"] < 2 * 8000 * 8
    pt.destroy(ctx)
    # ... except with contextual proposals, which need the spins in shared memory
    with pytest.raises(pt.PTError):
        pt.create_instances([I.ea_instance(20)], [I.geometric_betas(0.2, 2.0, 64)],
                            pt.Config(proposal_source=1, propose_every=2, context_sweeps=1),
                            prop_enabled=[[1] * 8 + [0] * 56])


def _graph(n, edges, h=None, clamp=None):
    e = np.array(edges, dtype=np.int32).reshape(-1, 3)
    return I.Instance(n, e[:, 0].copy(), e[:, 1].copy(), e[:, 2].copy(),
                      None if h is None else np.asarray(h, np.int32),
                      None if clamp is None else np.asarray(clamp, np.int8), 0)


@pytest.mark.parametrize("update", [0, 1])
def test_graph_without_edges_and_single_site(update):
    for inst in (_graph(5, [], h=[1, -2, 0, 3, -1]), _graph(1, [], h=[2])):
        betas = I.geometric_betas(0.3, 2.0, 6)
        cfg = pt.Config(update=update, seed=3)
        ctx = pt.create_instances([inst], [betas], cfg, instance_ids=[8])
        assert pt.info(ctx)["engine"] == "graph"
        pt.run_cycles(ctx, 25)
        o = O.Oracle(inst, betas, instance_id=8, update=update, seed=3)
        o.run_cycles(25)
        _same(ctx, 0, o)


def test_graph_with_every_spin_clamped():
    inst = _graph(4, [(0, 1, 1), (1, 2, -2), (2, 3, 1)], h=[0, 1, 0, -1], clamp=[1, -1, -1, 1])
    betas = I.geometric_betas(0.3, 2.0, 5)
    ctx = pt.create_instances([inst], [betas], pt.Config(update=1, seed=2), instance_ids=[1])
    pt.run_cycles(ctx, 10)
    o = O.Oracle(inst, betas, instance_id=1, update=1, seed=2)
    o.run_cycles(10)
    _same(ctx, 0, o)
    s, E = pt.read_state(ctx, 0)
    assert np.all(s == np.array([1, -1, -1, 1], np.int8)[None, :])
    assert len(set(E.tolist())) == 1                    # one configuration, one energy


def test_zero_length_calls_change_nothing():
    inst = I.ea_instance(4, index=6)
    betas = I.geometric_betas(0.2, 2.0, 8)
    ctx = pt.create_instances([inst], [betas], pt.Config(seed=4), instance_ids=[2])
    s0, E0 = pt.read_state(ctx, 0)
    pt.run_cycles(ctx, 0)
    pt.sweep(ctx, 0)
    s1, E1 = pt.read_state(ctx, 0)
    assert np.array_equal(s0, s1) and np.array_equal(E0, E1)
    c, _ = pt.read_counters(ctx, 0)
    assert list(c) == [0, 0, 0]


def test_empty_batch_rejected():
    with pytest.raises(pt.PTError):
        pt.create_instances([], [], pt.Config())


def test_pool_of_one_entry_proposed_every_sweep():
    inst = I.ea_instance(6, index=3)
    R, P = 10, 1
    betas = I.geometric_betas(0.1, 3.0, R)
    prop = [1] * (R - 1) + [0]
    cfg = pt.Config(seed=7, propose_every=1, propose_start=0, pool_size=P)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[5])
    o = O.Oracle(inst, betas, instance_id=5, prop_enabled=prop, propose_every=1, seed=7,
                 pool_size=P)
    for r in range(R):
        pool = I.random_configs(inst.n_spins, P, seed=31, index=r)
        pt.load_proposals(ctx, 0, r, pool)
        o.load_pool(r, pool)
    pt.run_cycles(ctx, 30)
    o.run_cycles(30)
    _same(ctx, 0, o)
    assert np.array_equal(pt.read_counters(ctx, 0)[1], o.cursors())
