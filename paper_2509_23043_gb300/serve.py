"""Continuous-batching TAPT server on one GPU, and time-to-target accounting.

Requests are lattice spin-glass instances that arrive over time. Each carries a proposal pool
made offline by PT runs of this library (excluded from timing, as bank generation is in the
paper's time-to-solution, Methods) and a reference lowest energy. The server keeps one
context of pre-sized slots (one size class per L); a request is admitted into a free slot of
its class when the device-memory budget allows. Its replica state and pool then stay on the
device and it runs, cycle after cycle, together with every other admitted request in the
same launches. When its best replica energy reaches the target, or the sweep budget is spent,
it retires and frees its slot. A request that can never be admitted (no slot class for its L,
or a footprint above the device-memory budget) is rejected at arrival; a request can be
cancelled, and one past its deadline retires unsolved, whether waiting or running.

Every request's random streams are keyed by its request id, and its counters start at zero
on admission, so its trajectory (and its sweeps-to-target) is the same alone or in the mix.

Time-to-solution follows the paper's definition of success within a run (Eq. for TTS and
Supplementary S5): here one run per request, success = reaching E_ref + 0.1% |E_ref|.

Admission by device memory is modelled: every slot's state and pool are allocated when the
server is built, and the budget caps the summed footprint (footprint_bytes) of the requests
admitted at once, so a request can wait for memory while a slot of its class is free.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import (Config, create_instances, destroy, energies, load_proposals_inst_packed,
               read_counters, read_proposals_packed, run_cycles, run_cycles_graph,
               capture_proposals, set_active, set_instance, read_state, read_walkers)


@dataclass
class Request:
    rid: int                    # request id; keys the random streams
    instance: object            # lattice instance (instances.Instance)
    betas: np.ndarray
    prop: list
    pool: np.ndarray | None     # uint32 [P][R][ceil(N/32)]
    e_ref: int                  # reference lowest energy
    arrival: float = 0.0        # seconds after the start of the stream
    deadline: float = math.inf  # seconds after arrival; past it the request retires unsolved
    admitted: float = math.nan
    finished: float = math.nan
    sweeps: int = -1            # sweeps from admission to the target (-1: not reached)
    best: int = 0
    status: str = "pending"     # then "solved", "budget", "rejected", "cancelled", "timeout"
    mem_waits: int = 0          # admission attempts refused by the device-memory budget
    final: tuple | None = None  # (spins [R][N], energies [R], walker of each slot) at retirement

    @property
    def L(self) -> int:
        return int(self.instance.lattice_L)

    @property
    def target(self) -> int:
        return int(math.floor(self.e_ref + 0.001 * abs(self.e_ref)))

    @property
    def tts(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Lattice:
    """A placeholder periodic L^3 lattice (all bonds +1) for a free slot."""
    L: int
    n_spins: int = 0
    edge_i: np.ndarray = field(default=None)
    edge_j: np.ndarray = field(default=None)
    edge_J: np.ndarray = field(default=None)
    h: None = None
    clamp: None = None
    lattice_L: int = 0

    def __post_init__(self):
        L = self.L
        n = np.arange(L ** 3)
        x, y, z = n % L, (n // L) % L, n // (L * L)
        nb = np.stack([((x + 1) % L) + L * (y + L * z), x + L * (((y + 1) % L) + L * z),
                       x + L * (y + L * ((z + 1) % L))], axis=1)
        self.n_spins = L ** 3
        self.lattice_L = L
        self.edge_i = np.repeat(n, 3).astype(np.int32)
        self.edge_j = nb.reshape(-1).astype(np.int32)
        self.edge_J = np.ones(3 * L ** 3, dtype=np.int32)


def footprint_bytes(L: int, R: int, P: int) -> int:
    """Device memory a slot of this shape holds: bit-packed state and its proposal pool."""
    N = L ** 3
    nw = (N + 31) // 32
    W = (R + 31) // 32
    return W * N * 4 + P * R * nw * 4 + N * 16


def make_pools(insts, betas, ids, P: int, burnin: int, gap: int, seed: int = 0x9001,
               stream=None) -> list[np.ndarray]:
    """Pools of P configurations per slot from one PT run per instance (this library):
    `burnin` sweeps, then a capture every `gap` sweeps. Returns uint32 [P][R][NW] each."""
    cfg_g = Config(seed=seed)
    gen = create_instances(insts, betas, cfg_g, instance_ids=[1_000_000 + i for i in ids],
                           stream=stream)
    dst = create_instances(insts, betas, Config(seed=seed, pool_size=P),
                           instance_ids=list(ids), stream=stream)
    run_cycles(gen, burnin)
    for e in range(P):
        run_cycles(gen, gap)
        capture_proposals(dst, gen, e)
    Rs = [len(b) for b in betas]
    nws = [(int(i.n_spins) + 31) // 32 for i in insts]
    slab = sum(R * nw for R, nw in zip(Rs, nws))
    words = np.zeros((P, slab), dtype=np.uint32)
    read_proposals_packed(dst, words, 0, P)
    out, off = [], 0
    for R, nw in zip(Rs, nws):
        out.append(np.ascontiguousarray(words[:, off:off + R * nw].reshape(P, R, nw)))
        off += R * nw
    destroy(gen)
    destroy(dst)
    return out


def host_energy(inst, spins) -> int:
    """E = -sum_edges J m_i m_j - sum_i h_i m_i of one +-1 configuration, recomputed on the
    host with numpy from the instance's edge list (Supplementary S4): an independent check of
    the energies the device reports."""
    m = np.asarray(spins, dtype=np.int64)
    E = -int(np.sum(np.asarray(inst.edge_J, np.int64) * m[inst.edge_i] * m[inst.edge_j]))
    if inst.h is not None:
        E -= int(np.dot(np.asarray(inst.h, np.int64), m))
    return E


def reference_energies(insts, betas, ids, sweeps: int, chunk: int = 1000, seed: int = 0x5EF,
                       runs: int = 1, stream=None, verify: bool = False) -> list[int]:
    """Lowest energy met by `runs` independent long PT runs of every instance (own random
    streams each, checked every `chunk` sweeps). With verify, the configuration that reached
    each best energy is read back and its energy recomputed on the host (host_energy), and a
    mismatch raises."""
    best = [10 ** 9] * len(insts)
    for run in range(runs):
        ctx = create_instances(insts, betas, Config(seed=seed + 0x1000 * run),
                               instance_ids=[2_000_000 + 100_000 * run + i for i in ids], stream=stream)
        done = 0
        while done < sweeps:
            n = min(chunk, sweeps - done)
            run_cycles(ctx, n)
            done += n
            for k, e in enumerate(energies(ctx)):
                lo = int(e.min())
                if lo < best[k]:
                    best[k] = lo
                    if verify:
                        spins, E = read_state(ctx, k)
                        r = int(np.argmin(E))
                        if host_energy(insts[k], spins[r]) != int(E[r]):
                            raise RuntimeError(f"instance {k}: reported energy {int(E[r])} is not "
                                               f"the configuration's ({host_energy(insts[k], spins[r])})")
        destroy(ctx)
    return best


class TaptServer:
    """Slots per lattice size L (all with R replicas and pools of P entries)."""

    def __init__(self, slots_per_L: dict[int, int], betas: np.ndarray, prop: list,
                 config: Config, hbm_budget: int | None = None, tick_cycles: int = 100,
                 use_graph: bool = True, keep_final: bool = False, stream=None):
        self.R = len(betas)
        self.cfg = config
        self.tick_cycles = tick_cycles
        self.use_graph = use_graph
        self.keep_final = keep_final
        self.slot_L, placeholders, ids = [], [], []
        for L, n in sorted(slots_per_L.items()):
            for j in range(n):
                self.slot_L.append(L)
                placeholders.append(_Lattice(L))
                ids.append(0xFFFF0000 + len(ids))
        self.ctx = create_instances(placeholders, [betas] * len(placeholders), config,
                                    prop_enabled=[prop] * len(placeholders), instance_ids=ids,
                                    stream=stream)
        for k in range(len(placeholders)):
            set_active(self.ctx, k, False)
        self.free = {L: [k for k, l in enumerate(self.slot_L) if l == L] for L in slots_per_L}
        self.active: dict[int, Request] = {}
        self.ticks_of: dict[int, int] = {}
        self.budget = hbm_budget
        self.used = 0
        self.peak_used = 0        # largest footprint admitted at once (bytes)
        self.peak_active = 0      # most requests in flight at once
        self.cancelled: set[int] = set()

    def cancel(self, rid: int) -> None:
        """Withdraw request `rid`: dropped if still waiting, retired at the next tick if running."""
        self.cancelled.add(rid)

    def fits(self, req: Request) -> bool:
        """Whether the request can ever be admitted: a slot class for its L, and a footprint
        within the device-memory budget."""
        return req.L in self.free and (self.budget is None or self._fp(req) <= self.budget)

    def _fp(self, req: Request) -> int:
        return footprint_bytes(req.L, self.R, self.cfg.pool_size)

    def try_admit(self, req: Request, now: float) -> bool:
        if not self.free.get(req.L):
            return False
        if self.budget is not None and self.used + self._fp(req) > self.budget:
            req.mem_waits += 1
            return False
        k = self.free[req.L].pop()
        set_instance(self.ctx, k, req.instance, req.betas, req.prop, instance_id=req.rid)
        if req.pool is not None:
            load_proposals_inst_packed(self.ctx, k, req.pool)
        self.active[k] = req
        self.ticks_of[k] = 0
        self.used += self._fp(req)
        self.peak_used = max(self.peak_used, self.used)
        self.peak_active = max(self.peak_active, len(self.active))
        req.admitted = now
        return True

    def _retire(self, k: int, req: Request, now: float, status: str) -> None:
        req.status = status
        req.finished = now
        if self.keep_final:
            spins, E = read_state(self.ctx, k)
            req.final = (spins, E, read_walkers(self.ctx, k))
        set_active(self.ctx, k, False)
        self.free[req.L].append(k)
        self.used -= self._fp(req)
        del self.active[k]

    def tick(self, now_fn, budget_sweeps: int) -> list[Request]:
        if not self.active:
            return []
        if self.use_graph:
            run_cycles_graph(self.ctx, self.tick_cycles)
        else:
            run_cycles(self.ctx, self.tick_cycles)
        E = energies(self.ctx)                      # synchronises: results of this tick
        now = now_fn()
        done = []
        for k, req in list(self.active.items()):
            self.ticks_of[k] += 1
            sw = self.ticks_of[k] * self.tick_cycles * self.cfg.sweeps_per_cycle
            req.best = int(E[k].min())
            if req.best <= req.target:
                req.sweeps = sw
                self._retire(k, req, now, "solved")
            elif sw >= budget_sweeps:
                req.budget_sweeps = sw
                self._retire(k, req, now, "budget")
            elif req.rid in self.cancelled:
                self._retire(k, req, now, "cancelled")
            elif now - req.arrival > req.deadline:
                self._retire(k, req, now, "timeout")
            else:
                continue
            done.append(req)
        return done

    def serve(self, requests: list[Request], budget_sweeps: int) -> list[Request]:
        """Admit requests at their arrival times (in order), run until all retire."""
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting: list[Request] = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        finished: list[Request] = []
        while pending or waiting or self.active:
            t = now()
            while pending and pending[0].arrival <= t:
                req = pending.pop(0)
                if not self.fits(req):                   # could never be admitted
                    req.status, req.finished = "rejected", t
                    finished.append(req)
                else:
                    waiting.append(req)
            still = []
            for req in waiting:
                if req.rid in self.cancelled or t - req.arrival > req.deadline:
                    req.status = "cancelled" if req.rid in self.cancelled else "timeout"
                    req.finished = t
                    finished.append(req)
                elif not self.try_admit(req, now()):
                    still.append(req)
            waiting = still
            if not self.active:
                if pending or waiting:
                    nxt = pending[0].arrival - now() if pending else 0.002
                    time.sleep(max(0.0, min(0.002, nxt)))
                continue
            finished += self.tick(now, budget_sweeps)
        return finished


def run_alone(req: Request, config: Config, budget_sweeps: int, tick_cycles: int = 100,
              keep_final: bool = False, stream=None) -> Request:
    """One request in its own context and launch (plain PT when config.propose_every == 0)."""
    ctx = create_instances([req.instance], [req.betas], config, prop_enabled=[req.prop],
                           instance_ids=[req.rid], stream=stream)
    if config.pool_size and req.pool is not None:
        load_proposals_inst_packed(ctx, 0, req.pool)
    t0 = time.perf_counter()
    sw = 0
    req.admitted = 0.0
    while True:
        run_cycles(ctx, tick_cycles)
        sw += tick_cycles * config.sweeps_per_cycle
        req.best = int(energies(ctx)[0].min())
        if req.best <= req.target or sw >= budget_sweeps:
            req.sweeps = sw if req.best <= req.target else -1
            req.budget_sweeps = sw
            req.status = "solved" if req.best <= req.target else "budget"
            break
    req.finished = time.perf_counter() - t0
    req.arrival = 0.0
    if keep_final:
        spins, E = read_state(ctx, 0)
        req.final = (spins, E, read_walkers(ctx, 0))
    destroy(ctx)
    return req


def summarize(reqs: list[Request]) -> dict:
    """Time to solution over the requests that ran (solved, or stopped by the sweep budget):
    p50/p99 in seconds and sweeps over all of them, a budget-limited request counted as
    censored at its budget (so a p99 that falls on a censored request is a lower bound, flagged
    by p99_censored); the same over the solved requests alone; the mean wait (arrival to
    admission), the mean service (admission to retirement) and the requests that waited for
    device memory; and the fitted TTS exponent k of log TTS = a + k L, and of
    log TTS = a + k N with N = L^3 (least squares over the per-L medians of the solved
    requests, as in TTS(n) = A exp(k n) of Supplementary S5)."""
    solved = [r for r in reqs if r.sweeps >= 0]
    ran = [r for r in reqs if r.status in ("solved", "budget")]
    out = {"requests": len(reqs), "solved": len(solved)}
    for st in ("budget", "rejected", "cancelled", "timeout"):
        n = sum(r.status == st for r in reqs)
        if n:
            out[st] = n
    out["censored"] = sum(r.status == "budget" for r in reqs)
    out["waited_for_memory"] = sum(r.mem_waits > 0 for r in reqs)
    if reqs:
        out["mean_wait_s"] = float(np.nanmean([r.admitted - r.arrival for r in reqs]))
        out["mean_service_s"] = float(np.nanmean([r.finished - r.admitted for r in reqs]))
    if ran:
        t = np.array([r.tts for r in ran])
        sw = np.array([r.sweeps if r.sweeps >= 0 else _ran_sweeps(r) for r in ran], dtype=np.float64)
        cens = np.array([r.status == "budget" for r in ran])
        out.update({"p50_s": float(np.percentile(t, 50)), "p99_s": float(np.percentile(t, 99)),
                    "p50_sweeps": float(np.percentile(sw, 50)),
                    "p99_sweeps": float(np.percentile(sw, 99)),
                    "p99_censored": bool(cens.any() and np.percentile(t, 99) >= t[cens].min())})
    if not solved:
        return out
    t = np.array([r.tts for r in solved])
    s = np.array([r.sweeps for r in solved], dtype=np.float64)
    out.update({"solved_p50_s": float(np.percentile(t, 50)), "solved_p99_s": float(np.percentile(t, 99)),
                "solved_p50_sweeps": float(np.percentile(s, 50)),
                "solved_p99_sweeps": float(np.percentile(s, 99))})
    Ls = sorted({r.L for r in solved})
    if len(Ls) >= 2:
        med = [float(np.median([r.tts for r in solved if r.L == L])) for L in Ls]
        medsw = [float(np.median([r.sweeps for r in solved if r.L == L])) for L in Ls]
        out["k_seconds_per_L"] = float(np.polyfit(Ls, np.log(med), 1)[0])
        out["k_sweeps_per_L"] = float(np.polyfit(Ls, np.log(medsw), 1)[0])
        Ns = [L ** 3 for L in Ls]                     # the same fit against the spin count
        out["k_seconds_per_N"] = float(np.polyfit(Ns, np.log(med), 1)[0])
        out["k_sweeps_per_N"] = float(np.polyfit(Ns, np.log(medsw), 1)[0])
    return out


def _ran_sweeps(r: Request) -> float:
    """Sweeps a budget-limited request ran: its budget (recorded when it retired)."""
    return float(getattr(r, "budget_sweeps", float("nan")))
