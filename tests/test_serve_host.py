"""The serving loop's host-side handling, on the CPU with a fake device backend (no GPU, no
fault): admission by slot class and device-memory budget, rejection of requests that can
never fit, cancellation, deadlines, and that the loop always ends."""
import math

import numpy as np
import pytest

from paper_2509_23043_gb300 import Config
from paper_2509_23043_gb300 import serve as S


class _FakeDevice:
    """Stands in for the library calls the server makes. Instance k's energies fall by one per
    tick from 0, so a request with target -t is solved after t ticks."""

    def __init__(self):
        self.n = 0
        self.ticks = {}
        self.active = {}

    def create_instances(self, insts, betas, cfg, prop_enabled=None, instance_ids=None, stream=None):
        self.n = len(insts)
        self.ticks = {k: 0 for k in range(self.n)}
        self.active = {k: True for k in range(self.n)}
        return object()

    def set_active(self, ctx, k, on):
        self.active[k] = bool(on)

    def set_instance(self, ctx, k, inst, betas, prop, instance_id=None):
        self.ticks[k] = 0                          # like pt_set_instance: fresh and active
        self.active[k] = True

    def load_proposals_inst_packed(self, ctx, k, pool):
        pass

    def run_cycles_graph(self, ctx, n):
        for k, on in self.active.items():
            if on:
                self.ticks[k] += 1

    def energies(self, ctx):
        return [np.array([-self.ticks[k]]) for k in range(self.n)]


@pytest.fixture
def fake(monkeypatch):
    dev = _FakeDevice()
    for name in ("create_instances", "set_active", "set_instance", "load_proposals_inst_packed",
                 "run_cycles_graph", "energies"):
        monkeypatch.setattr(S, name, getattr(dev, name))
    return dev


def _req(rid, L, ticks, arrival=0.0, deadline=math.inf):
    inst = S._Lattice(L)
    # target = floor(e_ref + 0.001 |e_ref|) = -ticks for these small references
    return S.Request(rid, inst, np.ones(4), [1, 1, 0, 0], None, -ticks, arrival=arrival,
                     deadline=deadline)


def _server(budget=None):
    return S.TaptServer({4: 2, 6: 1}, np.ones(4), [1, 1, 0, 0], Config(pool_size=8),
                        hbm_budget=budget, tick_cycles=10)


def test_requests_are_solved_in_slots_and_the_loop_ends(fake):
    srv = _server()
    reqs = [_req(k, 4, 3 + k) for k in range(5)] + [_req(9, 6, 2)]
    done = srv.serve(reqs, budget_sweeps=10_000)
    assert {r.rid: r.status for r in done} == {r.rid: "solved" for r in reqs}
    assert {r.rid: r.sweeps for r in done} == {r.rid: 10 * (-r.e_ref) for r in reqs}
    assert srv.peak_active <= 3 and not srv.active and srv.used == 0


def test_requests_that_can_never_fit_are_rejected_at_arrival(fake):
    fp4 = S.footprint_bytes(4, 4, 8)
    srv = _server(budget=fp4)                       # an L=6 request is above the budget
    reqs = [_req(1, 4, 2), _req(2, 6, 2), _req(3, 5, 2), _req(4, 4, 2)]
    done = {r.rid: r for r in srv.serve(reqs, budget_sweeps=10_000)}
    assert done[2].status == "rejected" and done[3].status == "rejected"   # budget, no L=5 slots
    assert done[1].status == "solved" and done[4].status == "solved"
    assert srv.peak_active == 1                     # the budget admits one L=4 slot at a time
    assert S.summarize(list(done.values()))["rejected"] == 2


def test_budget_and_deadline_and_cancellation(fake):
    srv = _server()
    srv.cancel(7)
    reqs = [_req(5, 4, 10 ** 6), _req(6, 4, 10 ** 6, deadline=0.0), _req(7, 6, 10 ** 6),
            _req(8, 4, 1)]
    done = {r.rid: r for r in srv.serve(reqs, budget_sweeps=50)}
    assert done[5].status == "budget" and done[5].sweeps == -1
    assert done[6].status == "timeout"
    assert done[7].status == "cancelled"
    assert done[8].status == "solved" and done[8].sweeps == 10
    s = S.summarize(list(done.values()))
    assert s["solved"] == 1 and s["budget"] == 1 and s["timeout"] == 1 and s["cancelled"] == 1


def test_summary_counts_budget_limited_requests_as_censored():
    # time to solution over every request that ran: one stopped by the sweep budget counts at
    # the budget (censored), so the p99 that falls on it is flagged as a lower bound
    from paper_2509_23043_gb300 import serve as S

    class _I:
        lattice_L = 6
    reqs = []
    for k in range(10):
        r = S.Request(k, _I(), None, None, None, -100, arrival=0.0)
        r.admitted, r.finished = 0.0, 1.0 + k
        if k < 8:
            r.status, r.sweeps = "solved", 100 * (k + 1)
        else:
            r.status, r.sweeps, r.budget_sweeps = "budget", -1, 5000
        reqs.append(r)
    out = S.summarize(reqs)
    assert out["solved"] == 8 and out["censored"] == 2
    assert out["p99_censored"] and out["p99_sweeps"] == 5000.0
    assert out["solved_p50_sweeps"] == 450.0
    assert out["p50_sweeps"] == float(np.percentile([100 * (k + 1) for k in range(8)] + [5000, 5000], 50))
