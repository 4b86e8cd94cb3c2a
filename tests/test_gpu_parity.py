"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element on
seeded inputs: spins, integer energies, walker labels (i.e. every exchange decision),
pool cursors, counters and acceptance statistics must be identical."""
import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2509_23043_gb300 as pt

pytestmark = pytest.mark.gpu


def _oracle(inst, betas, cfg, iid, prop=None):
    return O.Oracle(inst, betas, instance_id=iid, prop_enabled=prop, update=cfg.update,
                    sweeps_per_cycle=cfg.sweeps_per_cycle, propose_every=cfg.propose_every,
                    propose_start=cfg.propose_start, propose_stop=cfg.propose_stop,
                    seed=cfg.seed, pool_size=cfg.pool_size, colour_cap=cfg.colour_cap)


@pytest.mark.parametrize("bits,cap,update", [(4, 4, 1), (4, 8, 0), (8, 32, 1)])
def test_capped_colour_classes_match_oracle(bits, cap, update):
    # colour_cap: DSATUR classes rebalanced to at most `cap` free sites (ten classes of 4 and
    # five of 8 on the 4x4 multiplier's 40 free sites; five of 32 and one of 16 on the 8x8
    # multiplier's 176, the bench's setting); the chain follows the oracle's with the same
    # classes bit for bit
    mult = I.multiplier(bits)
    C = 11 * 13 if bits == 4 else 251 * 241
    inst = mult.instance(C)
    R, P = 16, 8
    betas = I.geometric_betas(0.05, 5.0, R)
    prop = [1] * 11 + [0] * 5
    cfg = pt.Config(update=update, seed=4242 + cap, propose_every=3, pool_size=P, colour_cap=cap)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[C])
    o = _oracle(inst, betas, cfg, C, prop)
    col, n = o.colouring()
    free = inst.clamp == 0
    sizes = [int(((col == c) & free).sum()) for c in range(n)]
    assert max(sizes) <= cap
    pools = [I.random_configs(inst.n_spins, P, seed=9, index=r) for r in range(R)]
    for r in range(R):
        pt.load_proposals(ctx, 0, r, pools[r])
        o.load_pool(r, pools[r])
    for chunk in (1, 7, 40):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _assert_same(ctx, 0, o, f"colour_cap {cap}")
    _stats_same(ctx, 0, o)


def _assert_same(ctx, k, o, what=""):
    s_g, E_g = pt.read_state(ctx, k)
    s_o, E_o, w_o = o.read()
    w_g = pt.read_walkers(ctx, k)
    assert np.array_equal(E_g, E_o), f"{what} energies differ"
    assert np.array_equal(w_g, w_o), f"{what} walker labels differ"
    assert np.array_equal(s_g, s_o), f"{what} spins differ"
    c_g, cur_g = pt.read_counters(ctx, k)
    assert np.array_equal(c_g, o.counters())
    if o.R and o.cursors().size:
        assert np.array_equal(cur_g, o.cursors())


def _stats_same(ctx, k, o):
    g = pt.read_stats(ctx, k)
    r = o.stats()
    for a, b in zip(g, r):
        assert np.array_equal(a, b)


def _ea_pool(inst, R, P, seed):
    return [I.random_configs(inst.n_spins, P, seed=seed, index=r) for r in range(R)]


@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("L,R", [(20, 40), (19, 72)])
def test_lattice_larger_than_shared_memory_matches_oracle(L, R, update):
    # L = 20 with two walker blocks (and L = 19, odd: three colours, with three blocks):
    # the {word, complement} spins and the neighbour table need more than the 227 KB of shared
    # memory a block can hold, so the instance runs on the kernels that keep them in global
    # memory; with a pool and proposals every 2 cycles the chain follows the oracle's bit for
    # bit, and the group's shared memory holds neither
    inst = I.ea_instance(L, index=L + R)
    P = 4
    betas = I.geometric_betas(0.2, 3.0, R)
    cfg = pt.Config(seed=0xB16 + L, sweeps_per_cycle=1, update=update, propose_every=2, pool_size=P)
    ctx = pt.create_instances([inst], [betas], cfg, instance_ids=[23])
    assert pt.info(ctx)["engine"] == "lattice"
    W, N = (R + 31) // 32, L ** 3
    assert pt.group_info(ctx)[0]["smem"] < W * N * 8          # the spins are not in shared memory
    o = _oracle(inst, betas, cfg, 23)
    pools = _ea_pool(inst, R, P, seed=L)
    for r in range(R):
        pt.load_proposals(ctx, 0, r, pools[r])
        o.load_pool(r, pools[r])
    _assert_same(ctx, 0, o, "initial")
    for chunk in (1, 2):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _assert_same(ctx, 0, o, f"global-memory lattice L={L} R={R} update={update}")
    _stats_same(ctx, 0, o)


@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("L,R", [(6, 16), (4, 32), (2, 5), (3, 8), (5, 33), (4, 70)])
def test_lattice_cycles_match_oracle(L, R, update):
    inst = I.ea_instance(L, index=L * 7 + R)
    betas = I.geometric_betas(0.2, 3.0, R)
    cfg = pt.Config(seed=0x5EED + L, sweeps_per_cycle=1, update=update)
    ctx = pt.create_instances([inst], [betas], cfg, instance_ids=[17])
    assert pt.info(ctx)["engine"] == "lattice"
    o = _oracle(inst, betas, cfg, 17)
    _assert_same(ctx, 0, o, "initial")
    for chunk in (1, 7, 40):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _assert_same(ctx, 0, o, f"after {chunk}")
    _stats_same(ctx, 0, o)


@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("M", [1, 3])
def test_lattice_tapt_with_pool_matches_oracle(M, update):
    L, R, P = 4, 12, 37
    inst = I.ea_instance(L, index=3)
    betas = I.geometric_betas(0.1, 3.0, R)
    prop = [1] * (R - 2) + [0, 0]
    cfg = pt.Config(seed=77, sweeps_per_cycle=M, propose_every=2, propose_start=4, pool_size=P,
                    update=update)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[5])
    o = _oracle(inst, betas, cfg, 5, prop)
    pools = _ea_pool(inst, R, P, 99)
    for r in range(R):
        pt.load_proposals(ctx, 0, r, pools[r])
        o.load_pool(r, pools[r])
    for chunk in (3, 10, 50):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _assert_same(ctx, 0, o, f"M={M}")
    _stats_same(ctx, 0, o)
    _, _, pa, pt_ = o.stats()
    assert pt_.sum() > 0 and pa.sum() > 0


def test_manual_api_sequence_matches_oracle():
    inst = I.ea_instance(4, index=8)
    R, P = 9, 16
    betas = I.geometric_betas(0.3, 2.5, R)
    prop = [1] * R
    cfg = pt.Config(seed=1234, pool_size=P)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[3])
    o = _oracle(inst, betas, cfg, 3, prop)
    pools = _ea_pool(inst, R, P, 5)
    for r in range(R):
        pt.load_proposals(ctx, 0, r, pools[r])
        o.load_pool(r, pools[r])
    for step in range(12):
        pt.sweep(ctx, 1 + step % 3); o.sweeps(1 + step % 3)
        if step % 2:
            pt.global_propose(ctx); o.propose()
        pt.exchange(ctx); o.exchange()
        _assert_same(ctx, 0, o, f"step {step}")


@pytest.mark.parametrize("update", [0, 1])
def test_ragged_lattice_batch_and_mix_invariance(update):
    Ls = [6, 4, 7, 2, 5, 8]
    Rs = [16, 24, 8, 3, 40, 32]
    insts = [I.ea_instance(L, index=100 + k) for k, L in enumerate(Ls)]
    betas = [I.geometric_betas(0.1, 3.0, R) for R in Rs]
    P = 8
    props = [[1] * (R - 1) + [0] for R in Rs]
    cfg = pt.Config(seed=2025, propose_every=3, pool_size=P, update=update)
    ids = [1000 + k for k in range(len(Ls))]
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=props, instance_ids=ids)
    pools = [_ea_pool(insts[k], Rs[k], P, 40 + k) for k in range(len(Ls))]
    for k in range(len(Ls)):
        for r in range(Rs[k]):
            pt.load_proposals(ctx, k, r, pools[k][r])
    pt.run_cycles(ctx, 25)
    for k in range(len(Ls)):
        o = _oracle(insts[k], betas[k], cfg, ids[k], props[k])
        for r in range(Rs[k]):
            o.load_pool(r, pools[k][r])
        o.run_cycles(25)
        _assert_same(ctx, k, o, f"instance {k}")
    # the same instance alone gives the same trajectory (random streams keyed by its id)
    alone = pt.create_instances([insts[2]], [betas[2]], cfg, prop_enabled=[props[2]], instance_ids=[ids[2]])
    for r in range(Rs[2]):
        pt.load_proposals(alone, 0, r, pools[2][r])
    pt.run_cycles(alone, 25)
    a, b = pt.read_state(alone, 0), pt.read_state(ctx, 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("update", [1, 0])
def test_multiplier_graph_matches_oracle(update):
    mult = I.multiplier(4)
    C = 11 * 13
    inst = mult.instance(C)
    R, P = 10, 24
    betas = I.geometric_betas(0.05, 5.0, R)
    prop = [1] * 7 + [0] * 3
    cfg = pt.Config(update=update, seed=31337, propose_every=2, pool_size=P)
    ctx = pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[C])
    assert pt.info(ctx)["engine"] == "graph"
    o = _oracle(inst, betas, cfg, C, prop)
    pools = [I.random_configs(inst.n_spins, P, seed=8, index=r) for r in range(R)]
    for r in range(R):
        pt.load_proposals(ctx, 0, r, pools[r])
        o.load_pool(r, pools[r])
    _assert_same(ctx, 0, o, "initial")
    for chunk in (1, 9, 60):
        pt.run_cycles(ctx, chunk)
        o.run_cycles(chunk)
        _assert_same(ctx, 0, o, f"graph update={update}")
    _stats_same(ctx, 0, o)


@pytest.mark.parametrize("engine", ["lattice", "graph"])
@pytest.mark.parametrize("L", [3, 4])
def test_lattice_gibbs_on_both_engines(L, engine):
    # a lattice runs on the bit-packed engine (bit-plane uniforms); the same couplings given
    # as a general graph run on the int8 engine (one uniform word per walker)
    inst = I.ea_instance(L, index=50 + L)
    if engine == "graph":
        inst = I.Instance(inst.n_spins, inst.edge_i, inst.edge_j, inst.edge_J, None, None, 0)
    R = 6
    betas = I.geometric_betas(0.2, 2.0, R)
    cfg = pt.Config(update=1, seed=9)
    ctx = pt.create_instances([inst], [betas], cfg, instance_ids=[L])
    assert pt.info(ctx)["engine"] == engine
    o = _oracle(inst, betas, cfg, L)
    assert o.bitplane == (engine == "lattice")
    pt.run_cycles(ctx, 30)
    o.run_cycles(30)
    _assert_same(ctx, 0, o)


def test_checkpoint_roundtrip_is_exact():
    inst = I.ea_instance(5, index=2)
    R, P = 7, 10
    betas = I.geometric_betas(0.2, 3.0, R)
    prop = [1] * R
    cfg = pt.Config(seed=4, propose_every=2, pool_size=P)
    pools = _ea_pool(inst, R, P, 3)
    mk = lambda: pt.create_instances([inst], [betas], cfg, prop_enabled=[prop], instance_ids=[9])
    a, b = mk(), mk()
    for ctx in (a, b):
        for r in range(R):
            pt.load_proposals(ctx, 0, r, pools[r])
    pt.run_cycles(a, 40)
    pt.run_cycles(b, 20)
    s, _ = pt.read_state(b, 0)
    w = pt.read_walkers(b, 0)
    c, cur = pt.read_counters(b, 0)
    d = mk()
    for r in range(R):
        pt.load_proposals(d, 0, r, pools[r])
    pt.write_state(d, 0, s, w, c, cur)
    pt.run_cycles(d, 20)
    for x, y in zip(pt.read_state(a, 0), pt.read_state(d, 0)):
        assert np.array_equal(x, y)
    assert np.array_equal(pt.read_walkers(a, 0), pt.read_walkers(d, 0))


def test_capture_proposals_builds_pool_from_state():
    inst = I.ea_instance(4, index=1)
    R = 6
    betas = I.geometric_betas(0.2, 3.0, R)
    src = pt.create_instances([inst], [betas], pt.Config(seed=1), instance_ids=[1])
    dst = pt.create_instances([inst], [betas], pt.Config(seed=2, pool_size=3), instance_ids=[2])
    pt.run_cycles(src, 10)
    pt.capture_proposals(dst, src, 1)
    s, _ = pt.read_state(src, 0)
    # dst has pool entries 0 and 2 unset (all spins -1) and entry 1 captured from src; two
    # proposal events (all slots enabled) then match the oracle given the same pool
    dst2 = pt.create_instances([inst], [betas], pt.Config(seed=2, pool_size=3),
                               prop_enabled=[[1] * R], instance_ids=[2])
    pt.capture_proposals(dst2, src, 1)
    o = O.Oracle(inst, betas, instance_id=2, seed=2, pool_size=3, prop_enabled=[1] * R)
    zero = -np.ones((1, inst.n_spins), np.int8)
    for r in range(R):
        o.load_pool(r, zero, 0)
        o.load_pool(r, s[r:r + 1], 1)
        o.load_pool(r, zero, 2)
    for _ in range(2):
        pt.global_propose(dst2)
        o.propose()
    _assert_same(dst2, 0, o, "captured pool")


def test_bad_inputs_rejected():
    inst = I.ea_instance(4)
    with pytest.raises(pt.PTError):
        pt.create_instances([inst], [[2.0, 1.0]], pt.Config())          # descending ladder
    with pytest.raises(pt.PTError):
        pt.create_instances([inst], [np.ones(200)], pt.Config())        # R > 128
    bad = I.Instance(inst.n_spins, inst.edge_i[::-1].copy(), inst.edge_j[::-1].copy(),
                     inst.edge_J.copy(), lattice_L=4)
    with pytest.raises(pt.PTError):
        pt.create_instances([bad], [[1.0]], pt.Config())                # non-canonical bonds
    ctx = pt.create_instances([inst], [[1.0, 2.0]], pt.Config(pool_size=2))
    with pytest.raises(pt.PTError):
        pt.load_proposals(ctx, 0, 0, np.ones((3, inst.n_spins), np.int8))  # beyond the pool
    with pytest.raises(pt.PTError):
        pt.read_state(ctx, 5)
