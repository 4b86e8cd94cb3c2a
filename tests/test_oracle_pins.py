"""Pins of the CPU oracle against facts fixed outside the oracle itself: published
known-answer vectors, the paper's gate tables and spin counts, closed forms, invariants and
brute-force Boltzmann distributions. Each test names the passage it follows."""
import itertools
import math
from pathlib import Path

import numpy as np
import pytest

import instances as I
import oracle as O

GOLDEN = Path(__file__).parent / "golden"


# ------------------------------------------------------------------ Philox (Salmon et al.)
def test_philox_known_answers():
    rows = [l.split() for l in (GOLDEN / "philox4x32_10_kat.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(t, 16) for t in row]
        out = O.philox(v[0:4], v[4:6])
        assert list(out) == v[6:10]


# ------------------------------------------------------------------ thresholds
def test_metropolis_threshold_closed_form_and_monotone():
    for beta in (0.05, 0.2, 1.0, 3.0):
        prev = 2 ** 32
        for dE in range(1, 40):
            T = O.metropolis_threshold(beta, dE)
            assert T == min(math.floor(math.exp(-beta * dE) * 2 ** 32), 2 ** 32 - 1)
            assert T <= prev
            prev = T
    assert O.metropolis_threshold(0.0, 4) == 2 ** 32 - 1  # capped


def test_gibbs_threshold_symmetry():
    # (1 + tanh(bI))/2 + (1 + tanh(-bI))/2 = 1, so T(I) + T(-I) is 2^32 up to flooring
    for beta in (0.05, 0.5, 1.7, 4.6):
        assert O.gibbs_threshold(beta, 0) == 2 ** 31
        for Iv in range(1, 30):
            s = O.gibbs_threshold(beta, Iv) + O.gibbs_threshold(beta, -Iv)
            assert 2 ** 32 - 2 <= s <= 2 ** 32


def test_accept_rule_probability():
    # accept iff u + 1 <= 2^32 e^x: the accepted set of u is {0 .. floor(2^32 e^x) - 1}
    for x in (-0.1, -1.0, -5.0, -20.0):
        k = math.floor(math.ldexp(math.exp(x), 32))
        assert O.accept(x, k - 1) and not O.accept(x, k)
    assert O.accept(0.0, 2 ** 32 - 1) and O.accept(3.0, 2 ** 32 - 1)
    assert not O.accept(-23.0, 0)  # 2^32 e^-23 < 1


# ------------------------------------------------------------------ energy
@pytest.mark.parametrize("L", [2, 3, 4, 5])
def test_ferromagnet_ground_state(L):
    inst = I.ea_instance(L, ferro=True)
    up = np.ones(inst.n_spins, np.int8)
    assert O.energy(inst, up) == -3 * L ** 3
    assert O.energy(inst, -up) == -3 * L ** 3


def test_gauge_invariance():
    g = np.random.default_rng(5)
    inst = I.ea_instance(5, index=3)
    for _ in range(5):
        tau = g.choice(np.array([-1, 1], np.int8), inst.n_spins)
        m = g.choice(np.array([-1, 1], np.int8), inst.n_spins)
        J2 = (inst.edge_J * tau[inst.edge_i] * tau[inst.edge_j]).astype(np.int32)
        g_inst = I.Instance(inst.n_spins, inst.edge_i, inst.edge_j, J2, lattice_L=5)
        assert O.energy(g_inst, (tau * m).astype(np.int8)) == O.energy(inst, m)


def test_single_flip_energy_change_matches_local_field():
    # dE of flipping spin i equals 2 m_i I_i with I_i = sum_j J_ij m_j + h_i (Methods)
    m8 = I.multiplier(3).instance()
    g = np.random.default_rng(1)
    m = g.choice(np.array([-1, 1], np.int8), m8.n_spins)
    for i in range(m8.n_spins):
        Ii = int(m8.h[i])
        for a, b, J in zip(m8.edge_i, m8.edge_j, m8.edge_J):
            if a == i:
                Ii += int(J) * int(m[b])
            elif b == i:
                Ii += int(J) * int(m[a])
        f = m.copy(); f[i] = -f[i]
        assert O.energy(m8, f) - O.energy(m8, m) == 2 * int(m[i]) * Ii


# ------------------------------------------------------------------ gate tables (S4)
def _gate_instance(Jd, h):
    n = len(h)
    keys = sorted(Jd)
    return I.Instance(n, np.array([k[0] for k in keys], np.int32),
                      np.array([k[1] for k in keys], np.int32),
                      np.array([Jd[k] for k in keys], np.int32), np.array(h, np.int32))


def test_and_gate_truth_table():
    # Fig. S7: states (A,B,C) = 0, 2, 4, 7 (binary order, A most significant) are the four
    # minimum-energy states; the hand value is E = -3, and (1,1,0) has E = +1.
    g = _gate_instance(I.AND_J, I.AND_H)
    E = {}
    for k in range(8):
        bits = [(k >> 2) & 1, (k >> 1) & 1, k & 1]
        E[k] = O.energy(g, np.array([2 * b - 1 for b in bits], np.int8))
    emin = min(E.values())
    assert emin == -3
    assert sorted(k for k, v in E.items() if v == emin) == [0, 2, 4, 7]
    assert E[6] == 1


def test_full_adder_truth_table():
    # Supplementary S4 / Fig. S2(a): the 8 rows with S + 2 Cout = A + B + Cin are exactly
    # the minimum-energy states of the 32.
    g = _gate_instance(I.FA_J, I.FA_H)
    E = {}
    for bits in itertools.product([0, 1], repeat=5):
        E[bits] = O.energy(g, np.array([2 * b - 1 for b in bits], np.int8))
    emin = min(E.values())
    valid = {b for b in E if b[3] + 2 * b[4] == b[0] + b[1] + b[2]}
    assert {b for b, v in E.items() if v == emin} == valid
    assert emin == -4


# ------------------------------------------------------------------ multiplier (S4, S5)
def test_multiplier_spin_counts():
    # N = 3/4 n^2 + 1/2 n (Supplementary S5) with n = 2w: 200/252/310/374/444 (Table S3)
    assert [I.multiplier(w).n_spins for w in (8, 9, 10, 11, 12)] == [200, 252, 310, 374, 444]
    for w in range(2, 13):
        n = 2 * w
        assert I.multiplier(w).n_spins == 3 * n * n // 4 + n // 2


def _forward_state(mult, a, b):
    """Spins of the circuit computing a*b forward (every gate in a valid row)."""
    N = mult.n_spins
    val = {}
    for k, s in enumerate(mult.A):
        val[s] = (a >> k) & 1
    for k, s in enumerate(mult.B):
        val[s] = (b >> k) & 1
    for z in mult.zeros:
        val[z] = 0
    for kind, ids in mult.gates:  # gates are listed in dependency order
        if kind == "AND":
            val[ids[2]] = val[ids[0]] & val[ids[1]]
        else:
            t = val[ids[0]] + val[ids[1]] + val[ids[2]]
            val[ids[3]] = t & 1
            val[ids[4]] = t >> 1
    return np.array([2 * val[i] - 1 for i in range(N)], np.int8)


def test_multiplier_forward_product_and_worked_example():
    # the paper's worked example C = 1,022,117 = 1009 x 1013 (Fig. 4(d)) on a 10-bit circuit
    for w, a, b in [(4, 13, 11), (8, 251, 241), (10, 1009, 1013)]:
        mult = I.multiplier(w)
        s = _forward_state(mult, a, b)
        c = sum(1 << k for k, sp in enumerate(mult.C) if s[sp] > 0)
        assert c == a * b
        e_gs = -3 * w * w - 4 * w * (w - 1)  # every gate at its minimum
        assert O.energy(mult.instance(a * b), s) == e_gs
    assert 1009 * 1013 == 1022117


@pytest.mark.parametrize("w,products", [(2, [2, 3, 6, 9]), (3, [15, 21])])
def test_multiplier_ground_states_factor(w, products):
    # With C clamped, the ground states are exactly the configurations whose A*B = C
    # (Fig. 4(a); success criterion A x B = C of the main text), by brute force.
    mult = I.multiplier(w)
    e_gs = -3 * w * w - 4 * w * (w - 1)
    for C in products:
        inst = mult.instance(C)
        free = np.nonzero(inst.clamp == 0)[0]
        nf = len(free)
        base = np.where(inst.clamp != 0, inst.clamp, 1).astype(np.int64)
        codes = np.arange(2 ** nf, dtype=np.int64)
        S = np.tile(base.astype(np.int8), (len(codes), 1))
        S[:, free] = (2 * ((codes[:, None] >> np.arange(nf)) & 1) - 1).astype(np.int8)
        E = np.zeros(len(codes), np.int32)
        for a, b, J in zip(inst.edge_i, inst.edge_j, inst.edge_J):
            E -= int(J) * (S[:, a] * S[:, b]).astype(np.int32)
        E -= (S.astype(np.int32) * inst.h[None, :]).sum(1, dtype=np.int32)
        assert E.min() == e_gs
        gs = S[E == e_gs]
        A = ((gs[:, mult.A] > 0) * (1 << np.arange(w))).sum(1)
        B = ((gs[:, mult.B] > 0) * (1 << np.arange(w))).sum(1)
        assert np.all(A * B == C)
        pairs = {(a, b) for a in range(2 ** w) for b in range(2 ** w) if a * b == C}
        assert set(zip(A.tolist(), B.tolist())) == pairs
        # spot check through the oracle's energy for one ground state
        assert O.energy(inst, gs[0].astype(np.int8)) == e_gs


# ------------------------------------------------------------------ colouring (Methods)
@pytest.mark.parametrize("w", [8, 9, 10, 11, 12])
def test_dsatur_five_colours_multiplier(w):
    # "Five colours are sufficient for all circuit sizes" (Methods, Graph coloring)
    mult = I.multiplier(w)
    free = I.Instance(mult.n_spins, mult.edge_i, mult.edge_j, mult.edge_J, mult.h)
    o = O.Oracle(free, [1.0], update=1)
    col, n = o.colouring()
    assert n <= 5
    assert np.all(col[mult.edge_i] != col[mult.edge_j])
    # the colouring is of the interaction graph, so clamping the product changes nothing
    col2, n2 = O.Oracle(mult.instance(143), [1.0], update=1).colouring()
    assert n2 == n and np.array_equal(col2, col)


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6, 7])
def test_lattice_colouring_proper(L):
    inst = I.ea_instance(L)
    col, n = O.Oracle(inst, [1.0]).colouring()
    assert n == (2 if L % 2 == 0 else 3)
    assert np.all(col[inst.edge_i] != col[inst.edge_j])


# ------------------------------------------------------------------ dynamics vs Boltzmann
def _states(N):
    codes = np.arange(2 ** N)
    return (2 * ((codes[:, None] >> np.arange(N)) & 1) - 1).astype(np.int64)


def _boltzmann(inst, beta):
    S = _states(inst.n_spins)
    h = np.zeros(inst.n_spins, np.int64) if inst.h is None else inst.h.astype(np.int64)
    E = -(inst.edge_J[None, :] * S[:, inst.edge_i] * S[:, inst.edge_j]).sum(1) - (h * S).sum(1)
    if inst.clamp is not None:
        ok = np.all((inst.clamp == 0)[None, :] | (S == inst.clamp[None, :]), axis=1)
    else:
        ok = np.ones(len(S), bool)
    w = np.where(ok, np.exp(-beta * (E - E[ok].min())), 0.0)
    return w / w.sum(), E


def _code(s):
    return int(((s > 0).astype(np.int64) << np.arange(len(s))).sum())


def _histogram(o, slot, n_cycles, burn=200, cycle=True):
    N = o.N
    h = np.zeros(2 ** N)
    weights = 1 << np.arange(N)
    step = o.run_cycles if cycle else o.sweeps
    step(burn)
    for _ in range(n_cycles):
        step(1)
        s, _, _ = o.read()
        h[int(((s[slot] > 0) * weights).sum())] += 1
    return h / h.sum()


def _tv(p, q):
    return 0.5 * np.abs(p - q).sum()


def _assert_matches(p, q, n, E=None):
    """q (an empirical histogram over n correlated samples) agrees with p: the total
    variation must sit within 4x the sampling noise expected from n/3 independent draws,
    and, when energies are given, the energy histogram must agree to within 0.02."""
    n_eff = n / 3.0
    noise = 0.5 * np.sum(np.sqrt(2.0 * p * (1.0 - p) / (np.pi * n_eff)))
    assert _tv(p, q) < 4.0 * noise + 0.005, (_tv(p, q), noise)
    if E is not None:
        levels = np.unique(E)
        pe = np.array([p[E == e].sum() for e in levels])
        qe = np.array([q[E == e].sum() for e in levels])
        assert _tv(pe, qe) < 0.02, (pe, qe)


@pytest.mark.parametrize("update,bitplane", [(0, True), (1, True), (0, False), (1, False)])
def test_single_replica_samples_boltzmann_2x2x2(update, bitplane):
    # On the 2x2x2 lattice (256 states) a long single-temperature run reproduces the exact
    # Boltzmann law; a dropped term or a wrong sign in the update would not. Both rules, with
    # the bit-plane uniforms (the lattice) and with one word per walker (the same couplings
    # given as a general graph).
    inst = I.ea_instance(2, index=7)
    if not bitplane:
        inst = I.Instance(inst.n_spins, inst.edge_i, inst.edge_j, inst.edge_J, None, None, 0)
    beta = 0.45
    o = O.Oracle(inst, [beta], update=update, seed=11)
    assert o.bitplane == bitplane
    p, E = _boltzmann(inst, beta)
    q = _histogram(o, 0, 60000)
    _assert_matches(p, q, 60000, E)


def test_field_and_clamps_sample_boltzmann():
    # word layout, Metropolis, fields and clamps: a 3-bit multiplier with C clamped to 6
    mult = I.multiplier(2)
    inst = mult.instance(6)
    beta = 0.6
    for update in (0, 1):
        o = O.Oracle(inst, [beta], update=update, seed=3)
        p, E = _boltzmann(inst, beta)
        q = _histogram(o, 0, 60000)
        _assert_matches(p, q, 60000, E)


def test_parallel_tempering_marginals_match_boltzmann():
    # PT (sweeps + alternating exchanges) leaves the product of Boltzmann laws invariant
    # (Supplementary S2, W_swap), so each slot's marginal is pi_{beta_r}.
    inst = I.ea_instance(2, index=2)
    betas = np.array([0.2, 0.5, 1.0])
    o = O.Oracle(inst, betas, seed=5)
    N = inst.n_spins
    hist = np.zeros((3, 2 ** N))
    weights = 1 << np.arange(N)
    o.run_cycles(200)
    for _ in range(40000):
        o.run_cycles(1)
        s, E, _ = o.read()
        for r in range(3):
            hist[r, int(((s[r] > 0) * weights).sum())] += 1
    for r in range(3):
        p, E = _boltzmann(inst, betas[r])
        _assert_matches(p, hist[r] / hist[r].sum(), 40000, E)
    sa, st, _, _ = o.stats()
    assert np.all(st > 0) and np.all(sa > 0) and np.all(sa <= st)


def test_uniform_pool_proposals_keep_boltzmann():
    # A uniformly random pool is a symmetric independent proposal, for which the DeltaE-only
    # rule is the exact Metropolis-Hastings rule (Supplementary S2, Eq. for A_beta), so the
    # Boltzmann law stays invariant.
    inst = I.ea_instance(2, index=4)
    betas = np.array([0.3, 0.8])
    P = 4096
    o = O.Oracle(inst, betas, prop_enabled=[1, 1], propose_every=1, seed=9, pool_size=P)
    for r in range(2):
        o.load_pool(r, I.random_configs(inst.n_spins, P, index=r))
    N = inst.n_spins
    hist = np.zeros((2, 2 ** N))
    weights = 1 << np.arange(N)
    o.run_cycles(100)
    for _ in range(40000):
        o.run_cycles(1)
        s, _, _ = o.read()
        for r in range(2):
            hist[r, int(((s[r] > 0) * weights).sum())] += 1
    for r in range(2):
        p, E = _boltzmann(inst, betas[r])
        _assert_matches(p, hist[r] / hist[r].sum(), 40000, E)
    _, _, pa, pt = o.stats()
    assert np.all(pt > 0) and np.all(pa > 0)


def test_energies_recomputed_match_configurations():
    inst = I.ea_instance(4, index=1)
    o = O.Oracle(inst, I.geometric_betas(0.2, 2.0, 5), seed=1)
    o.run_cycles(20)
    s, E, w = o.read()
    for r in range(5):
        assert E[r] == O.energy(inst, s[r])
    assert sorted(w.tolist()) == list(range(5))


def test_checkpoint_resume_is_exact():
    inst = I.ea_instance(3, index=0)
    betas = I.geometric_betas(0.1, 3.0, 4)
    P = 16
    pools = [I.random_configs(inst.n_spins, P, index=10 + r) for r in range(4)]
    kw = dict(prop_enabled=[1, 1, 1, 0], propose_every=3, propose_start=5, seed=77, pool_size=P)
    a = O.Oracle(inst, betas, **kw)
    for r in range(4):
        a.load_pool(r, pools[r])
    a.run_cycles(40)
    b = O.Oracle(inst, betas, **kw)
    for r in range(4):
        b.load_pool(r, pools[r])
    b.run_cycles(20)
    s, E, w = b.read()
    cnt, cur = b.counters(), b.cursors()
    c = O.Oracle(inst, betas, **kw)
    for r in range(4):
        c.load_pool(r, pools[r])
    c.write(s, w)
    c.set_counters(cnt, cur)
    c.run_cycles(20)
    for x, y in zip(a.read(), c.read()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("log2", [1, 2, 3])
def test_contextual_proposal_keeps_the_stated_fraction(log2):
    # Supplementary S3 contextual proposals: at beta = 0 every refilled spin flips (Metropolis
    # at beta = 0 accepts every move) and every proposal is accepted, so one proposal event
    # flips exactly the spins that were not kept: a fraction 1 - 2^-log2 of them.
    inst = I.ea_instance(10, index=3)
    o = O.Oracle(inst, [0.0, 0.0], prop_enabled=[1, 1], seed=17, proposal_source=1,
                 context_log2=log2, context_sweeps=1)
    changed, total = 0, 0
    for _ in range(20):
        before, _, _ = o.read()
        o.propose()
        after, _, _ = o.read()
        changed += int((before != after).sum())
        total += before.size
    f = changed / total
    expect = 1.0 - 2.0 ** -log2
    assert abs(f - expect) < 4 * np.sqrt(expect * (1 - expect) / total), (f, expect)


def test_always_accepted_contextual_proposals_keep_boltzmann():
    # Copying a replica, freezing a random subset chosen independently of the state and
    # running Metropolis sweeps on the rest leaves pi_beta invariant, so with every proposal
    # accepted (proposal_rule 1) the slot marginals stay Boltzmann. A mistake in the refill
    # (a wrong sign, a wrong beta, a frozen spin moved) would not.
    inst = I.ea_instance(2, index=5)
    betas = np.array([0.35, 0.9])
    o = O.Oracle(inst, betas, prop_enabled=[1, 1], propose_every=1, seed=23,
                 proposal_rule=1, proposal_source=1, context_log2=1, context_sweeps=2)
    N = inst.n_spins
    hist = np.zeros((2, 2 ** N))
    weights = 1 << np.arange(N)
    o.run_cycles(200)
    for _ in range(40000):
        o.run_cycles(1)
        s, _, _ = o.read()
        for r in range(2):
            hist[r, int(((s[r] > 0) * weights).sum())] += 1
    for r in range(2):
        p, E = _boltzmann(inst, betas[r])
        _assert_matches(p, hist[r] / hist[r].sum(), 40000, E)
    _, _, pa, pt_ = o.stats()
    assert np.array_equal(pa, pt_) and pt_[0] > 0


# ------------------------------------------------------------------ proposal schedule
def _proposal_sweeps(M, every, start, stop, n_cycles):
    """Sweep counts s at the end of the cycles after which the oracle held a proposal event,
    observed one cycle at a time through its event counter."""
    inst = I.ea_instance(2, index=1)
    o = O.Oracle(inst, [0.3, 0.9], prop_enabled=[1, 1], sweeps_per_cycle=M,
                 propose_every=every, propose_start=start, propose_stop=stop, seed=3,
                 pool_size=1)
    for r in range(2):
        o.load_pool(r, I.random_configs(inst.n_spins, 1, index=r))
    seen, prev = [], 0
    for _ in range(n_cycles):
        o.run_cycles(1)
        sweeps, _, n_prop = (int(v) for v in o.counters())
        assert n_prop - prev in (0, 1)
        if n_prop > prev:
            seen.append(sweeps)
        prev = n_prop
    _, _, pa, pt_ = o.stats()
    assert list(pt_) == [len(seen)] * 2           # every enabled slot attempts once per event
    return seen


@pytest.mark.parametrize("M,every,start,stop,n_cycles,expected", [
    # Fig. 3: proposals from 100 MCS on, every sweep; the first event follows sweep 100
    (1, 1, 100, 0, 104, [100, 101, 102, 103, 104]),
    # the benchmark workloads: every 10 sweeps from sweep 100
    (1, 10, 100, 0, 131, [100, 110, 120, 130]),
    # Fig. S3: proposals only during the first 100 MCS; sweep 100 itself is the last
    (1, 1, 0, 100, 103, list(range(1, 101))),
    # three sweeps per cycle: the cycle ends at s = 3, 6, 9, ...; every 6 sweeps from 0
    (3, 6, 0, 0, 7, [6, 12, 18]),
    # two sweeps per cycle never end at an odd s, so start 3 with every 4 is never due
    (2, 4, 3, 15, 10, []),
    # a window of one sweep: start = stop = 5
    (1, 5, 5, 5, 20, [5]),
    # every = 0 disables proposals
    (1, 0, 0, 0, 12, []),
])
def test_proposal_schedule_event_times(M, every, start, stop, n_cycles, expected):
    # Algorithm 1 proposes every `every` sweeps once `start` sweeps are done, until `stop`
    # (Fig. 3, Fig. S3); the expected event times are listed by hand, so an off-by-one at
    # start or stop (s > start, s < stop) or a schedule counted in cycles rather than sweeps
    # fails one of these cases.
    assert _proposal_sweeps(M, every, start, stop, n_cycles) == expected


# ------------------------------------------------------------------ initial draw
def test_initial_replicas_are_uniform_and_independent():
    # Algorithm 1 starts every replica from a uniformly random configuration: spins are
    # independent fair +-1 draws. Over 64 instances x 64 walkers x 64 sites, the mean spin,
    # the mean of every walker lane, and the pair products of neighbouring walkers, walkers
    # one word apart, neighbouring sites and consecutive instance ids all sit within 5
    # standard deviations of 0 (false-failure probability below 6e-7 per check). A constant,
    # biased or shared draw fails.
    L, R, n_inst = 4, 64, 64
    inst = I.ea_instance(L, index=0)
    S = np.zeros((n_inst, R, inst.n_spins), np.float64)
    for k in range(n_inst):
        o = O.Oracle(inst, I.geometric_betas(0.1, 3.0, R), instance_id=1000 + k, seed=0x51)
        s, _, w = o.read()
        assert list(w) == list(range(R))            # slot r starts with walker r
        S[k] = s
    n = S.size
    assert abs(S.mean()) < 5 / np.sqrt(n)
    lane = S.mean(axis=(0, 2))                      # per walker, over instances and sites
    assert np.all(np.abs(lane) < 5 / np.sqrt(n_inst * inst.n_spins))
    pairs = {
        "walker w, w+1": S[:, :-1, :] * S[:, 1:, :],
        "walker w, w+32": S[:, :-32, :] * S[:, 32:, :],
        "site i, i+1": S[:, :, :-1] * S[:, :, 1:],
        "instance k, k+1": S[:-1] * S[1:],
    }
    for name, prod in pairs.items():
        assert abs(prod.mean()) < 5 / np.sqrt(prod.size), name


def test_initial_state_respects_clamps():
    # Algorithm 1 with clamped spins (Supplementary S4: product bits of the multiplier):
    # clamped sites start at their clamp value in every replica, free sites are drawn.
    mult = I.multiplier(4)
    inst = mult.instance(143)
    o = O.Oracle(inst, I.geometric_betas(0.05, 5.0, 40), seed=9)
    s, E, _ = o.read()
    cl = inst.clamp
    assert np.all(s[:, cl != 0] == cl[cl != 0])
    free = s[:, cl == 0].astype(np.float64)
    assert abs(free.mean()) < 5 / np.sqrt(free.size)
    for r in range(s.shape[0]):
        assert E[r] == O.energy(inst, s[r])


def _free_adjacent_same_colour(inst, col):
    free = inst.clamp == 0 if inst.clamp is not None else np.ones(inst.n_spins, bool)
    ei, ej = np.asarray(inst.edge_i), np.asarray(inst.edge_j)
    both = free[ei] & free[ej]
    return bool(np.any(col[ei][both] == col[ej][both]))


@pytest.mark.parametrize("cap", [1, 3, 8, 32])
def test_capped_colouring_is_proper_and_within_cap(cap):
    # colour_cap: every class is an independent set of free sites (a valid parallel update),
    # holds at most cap free sites where the graph allows it, and no colour is left empty.
    # With cap 1 every free site is a class of its own; at caps that DSATUR's classes already
    # meet the colouring is DSATUR's.
    mult = I.multiplier(4)
    inst = mult.instance(11 * 13)
    free = inst.clamp == 0
    base, n0 = O.Oracle(inst, I.geometric_betas(0.1, 2.0, 4), update=1).colouring()
    col, n = O.Oracle(inst, I.geometric_betas(0.1, 2.0, 4), update=1, colour_cap=cap).colouring()
    assert not _free_adjacent_same_colour(inst, col)
    sizes = [int(((col == c) & free).sum()) for c in range(n)]
    assert max(sizes) <= cap
    assert sorted(set(col.tolist())) == list(range(n))
    if cap == 1:
        assert all(s <= 1 for s in sizes) and sum(sizes) == int(free.sum())
    if cap >= max(int(((base == c) & free).sum()) for c in range(n0)):
        assert np.array_equal(col, base) and n == n0


def test_capped_colouring_keeps_boltzmann_on_a_small_graph():
    # the capped sweep is still a product of Gibbs updates over independent sets: a long Gibbs
    # run of the oracle at one temperature on a 5-spin frustrated graph with cap 1 (five
    # single-site classes) reproduces the exact Boltzmann law of its 32 states
    ei = np.array([0, 0, 1, 1, 2, 3, 0], np.int32)
    ej = np.array([1, 2, 2, 3, 3, 4, 4], np.int32)
    eJ = np.array([1, -2, 1, 1, -1, 2, 1], np.int32)
    h = np.array([1, 0, -1, 0, 1], np.int32)
    inst = I.Instance(n_spins=5, edge_i=ei, edge_j=ej, edge_J=eJ, h=h, clamp=np.zeros(5, np.int8))
    beta = 0.4
    o = O.Oracle(inst, [beta], update=1, seed=11, colour_cap=1)
    col, n = o.colouring()
    assert n == 5 and sorted(col.tolist()) == [0, 1, 2, 3, 4]
    states = np.array([[1 if (k >> (4 - i)) & 1 else -1 for i in range(5)] for k in range(32)], np.int8)
    E = np.array([O.energy(inst, s) for s in states], float)
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    counts = np.zeros(32)
    for _ in range(20000):
        o.sweeps(1)
        s = o.read()[0][0]
        counts[int(((s > 0).astype(int) << np.arange(4, -1, -1)).sum())] += 1
    q = counts / counts.sum()
    assert 0.5 * np.abs(q - p).sum() < 0.02
