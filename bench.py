#!/usr/bin/env python
"""Throughput benchmark of batched TAPT (arXiv 2509.23043, Algorithm 1) on GB300.

Workload (the batched-TAPT configuration): 256 periodic 3D Edwards-Anderson +-J instances,
L = 10 (1000 spins), J = +-1 with p = 0.5 from the seed, no field; 32 temperature slots,
beta geometric 0.1 -> 3.0; Metropolis checkerboard sweeps, one exchange event per sweep
(M = 1); global proposals every 10 sweeps (from sweep 100) on the 30 hottest slots, drawn
from device pools of 1024 configurations per slot per instance that PT runs of this library
produce before timing (untimed); spins bit-packed 32 walkers per uint32; FP64 acceptance of
exchanges and proposals.

One step = 100 cycles of Algorithm 1 over the whole batch (100 sweeps, 100 energy
evaluations, 10 proposal events, 100 exchange events) = 8.192e8 spin-flip attempts.
Metric: spin-flip attempts per ns (one attempt = one free-spin update decision).

  python bench.py [--gpus N --steps K --warmup W]        # our CUDA path
  python bench.py --impl reference                        # the CPU oracle (reference arm)
Under torchrun (N > 1) the instances are sharded across ranks (weak scaling: each rank runs
its own 256 instances); there is no collective in the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "spin-flip attempts/ns; p50/p99 time-to-target of batched served TAPT vs plain PT"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# The integer ALU pipe (logic, add, shift, compare) takes 2 warp instructions per clock per
# SM, i.e. 64 lanes: ncu reports the pipe's share of its peak, and against the SM's issue
# rate (4 warp instructions per clock) that peak is half the issue rate. Multiplies run on
# the separate FMA pipe and are not counted against it.
ALU_LANES_PER_SM = 64


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--update", choices=("metropolis", "gibbs"), default="metropolis",
                   help="local rule of the main workload (Metropolis, the benchmark's; Gibbs, "
                        "the paper's)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--instances", type=int, default=256)
    p.add_argument("--L", type=int, default=10)
    p.add_argument("--R", type=int, default=32)
    p.add_argument("--sweeps-per-step", type=int, default=100)
    p.add_argument("--pool-size", type=int, default=1024)
    # pools from a 10^6-sweep PT run per instance: 5e5 burn-in, then 1024 captures 488 apart
    p.add_argument("--pool-burnin", type=int, default=500_000)
    p.add_argument("--pool-gap", type=int, default=488)
    p.add_argument("--threads", type=int, default=0)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-configs", action="store_true")
    p.add_argument("--workloads", default="plain,engines,ragged,factor,ladder,large,context,tts,former",
                   help="other workloads to measure after the main one")
    p.add_argument("--factor-sweeps", type=int, default=20000)
    p.add_argument("--factor-pool-size", type=int, default=512)
    p.add_argument("--factor-pool-burnin", type=int, default=100_000)
    p.add_argument("--factor-pool-gap", type=int, default=25)
    p.add_argument("--serve-requests", type=int, default=66)
    p.add_argument("--serve-L", default="6,7,8,9,10,11,12,13,14,15,16")
    p.add_argument("--serve-budget", type=int, default=1_000_000)
    p.add_argument("--serve-ref-runs", type=int, default=4)
    p.add_argument("--serve-ref-sweeps", type=int, default=1_000_000)
    p.add_argument("--serve-gap-ms", type=float, default=4.0)
    p.add_argument("--serve-load", type=float, default=0.7,
                   help="offered load as a fraction of the served TAPT capacity (the completion "
                        "rate with every request submitted at once); 0 keeps --serve-gap-ms")
    p.add_argument("--serve-pool-burnin", type=int, default=100_000)
    p.add_argument("--serve-pool-gap", type=int, default=100)
    p.add_argument("--serve-hbm-frac", type=float, default=0.5,
                   help="device-memory budget of admitted requests, as a fraction of all slots")
    p.add_argument("--profile-case", choices=("lattice", "lattice-gibbs", "graph", "former", "former-sample"),
                   help="run one small case for a profiler capture and exit (no timing, no JSON)")
    p.add_argument("--cpu-sample-instances", type=int, default=16)
    p.add_argument("--cpu-sample-sweeps", type=int, default=60)
    return p.parse_args()


# ------------------------------------------------------------------------------ workload
def workload(args, first: int, count: int):
    import instances as I
    insts = [I.ea_instance(args.L, seed=I.MASTER_SEED, index=first + k) for k in range(count)]
    betas = [I.geometric_betas(0.1, 3.0, args.R) for _ in range(count)]
    prop = [[1] * (args.R - 2) + [0, 0] for _ in range(count)]
    ids = [first + k for k in range(count)]
    return insts, betas, prop, ids


def workload_name(args) -> str:
    rule = "" if args.update == "metropolis" else ", Gibbs moves"
    return (f"batched TAPT: {args.instances} EA +-J instances per GPU, L={args.L} "
            f"(N={args.L ** 3}), R={args.R} beta 0.1->3.0 geometric, proposals every 10 sweeps "
            f"on {args.R - 2} slots from pools of {args.pool_size}, {args.sweeps_per_step} "
            f"cycles per step{rule}")


def update_rule(args) -> int:
    return 1 if args.update == "gibbs" else 0


def make_config(args, pool_size):
    import paper_2509_23043_gb300 as pt
    return pt.Config(update=update_rule(args), sweeps_per_cycle=1, propose_every=10,
                     propose_start=100, pool_size=pool_size, seed=0x7A972509,
                     threads_per_block=args.threads)


def build_pools(args, insts, betas, prop, ids, ctx):
    """Pools from PT runs of the method itself: a separate batch (other random streams)
    burns in, then its slot configurations are captured every `gap` sweeps."""
    import paper_2509_23043_gb300 as pt
    cfg = pt.Config(seed=0x9001, sweeps_per_cycle=1, threads_per_block=args.threads,
                    update=update_rule(args))
    gen = pt.create_instances(insts, betas, cfg, instance_ids=[1_000_000 + i for i in ids])
    pt.run_cycles(gen, args.pool_burnin)
    for e in range(args.pool_size):
        pt.run_cycles(gen, args.pool_gap)
        pt.capture_proposals(ctx, gen, e)
    pt.destroy(gen)


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []          # (monotonic time of arrival, fields)
        self.proc = None
        self.window = None      # (start, end) of the timed region

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.monotonic(), [t.strip() for t in line.split(",")]))

    def wait_first(self, timeout=3.0):
        """Block until the first sample has arrived, so that sampling covers the timed region."""
        t0 = time.monotonic()
        while self.proc and not self.rows and time.monotonic() - t0 < timeout:
            time.sleep(0.01)

    def mark(self, start, end):
        self.window = (start, end)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [r for _, r in self.rows]
        if self.window:
            # samples that arrived during the timed region (each reports the state at most one
            # sampling period earlier), else the one just after it
            a, b = self.window
            inside = [r for t, r in self.rows if a <= t <= b + 0.2]
            later = [r for t, r in self.rows if t > b]
            rows = inside or later[:1] or rows
        sm = [float(r[0]) for r in rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 8:
                continue
            for k, nm in enumerate(names):
                if r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ roofline model
def plane_blocks_of(ctx, k, inst, update):
    """Expected plane blocks per word of instance k of a lattice context in its current state:
    a word (site, walker block) of 32 walkers needs plane blocks (4 planes = one Philox call)
    until each of its comparing walkers is decided, each plane deciding a walker with
    probability 1/2. The comparing walkers are those with dE > 0 (Metropolis) or all (Gibbs)."""
    import paper_2509_23043_gb300 as pt
    s, _ = pt.read_state(ctx, k)                 # [R][N] slot order
    walker = pt.read_walkers(ctx, k)             # walker of each slot
    L = int(inst.lattice_L)
    J = np.zeros((L ** 3, 6), np.int64)
    nb = np.zeros((L ** 3, 6), np.int64)
    for e, (a, b, j) in enumerate(zip(inst.edge_i, inst.edge_j, inst.edge_J)):
        d = e % 3
        J[a, 2 * d], nb[a, 2 * d] = j, b
        J[b, 2 * d + 1], nb[b, 2 * d + 1] = j, a
    unsat = (J[None, :, :] * s[:, :, None] * s[:, nb] < 0).sum(-1)   # [R][N]
    cmp = (unsat <= 2) if update == "metropolis" else np.ones_like(unsat, dtype=bool)
    per_word = []
    for wb in range((s.shape[0] + 31) // 32):
        in_block = (walker // 32) == wb
        per_word.append(blocks_for(cmp[in_block].sum(0)))
    return float(np.mean(np.concatenate(per_word)))


def expected_plane_blocks(ctx, args, sample=4):
    """Algorithmic random-number work of the bit-plane compare, averaged over the words of a
    state sample of the benchmark workload's first instances."""
    import instances as I
    return float(np.mean([plane_blocks_of(ctx, k, I.ea_instance(args.L, index=k), args.update)
                          for k in range(min(sample, ctx.n))]))


def blocks_for(n_und) -> np.ndarray:
    """Expected plane blocks of a word whose n_und walkers compare a uniform u with their
    thresholds MSB first: block k (4 planes) is needed iff some walker is still undecided
    after 4k planes, which for one walker has probability 2^-4k (u uniform); none for
    n_und = 0."""
    n = np.asarray(n_und, dtype=np.float64)
    b = np.zeros_like(n)
    for q in range(8):
        b += np.where(n > 0, 1.0 - (1.0 - 2.0 ** (-4 * q)) ** n, 0.0)
    return b


def alu_ops_per_word(e_blocks: float, gibbs: bool = False) -> float:
    """Algorithmic integer-ALU operations of one bit-sliced word update (32 attempts):
    6 three-input XORs (bond test) + 8 (bit-sliced adder) + 2 (class masks) + 2 (flip)
    + 4.5 (energy count in the last colour, half the words) + per plane block: 20 (the
    three-input XORs of Philox4x32-10's 10 rounds; its 20 wide multiplies run on the FMA pipe)
    + 4 planes x 5 for the compare the Metropolis kernel performs (2 to pick the class
    threshold, 3 to compare one plane). Gibbs: 4 for the class q and 1 for the flip instead of
    the class masks and flip, and per block 4 x 6 to pick each plane's threshold by a six-mux
    tree plus 9 for the chained compare of the four planes (4 steps for the decided-below bit,
    4 for the still-undecided mask, 1 to merge), the compare the Gibbs kernel performs."""
    if gibbs:
        return 6 + 8 + 4 + 1 + 4.5 + e_blocks * (20 + 24 + 9)
    return 6 + 8 + 2 + 2 + 4.5 + e_blocks * (20 + 20)


def smem_bytes_per_word(e_blocks: float, gibbs: bool = False) -> float:
    """Algorithmic shared-memory bytes of one bit-sliced word update (32 attempts): the 16 B
    table entry, the own word and six neighbour words (4 B each), the 4 planes x 3 threshold
    words of every plane block drawn (48 B per block; Gibbs: 4 x 7 words, 112 B), and the 8 B
    word-and-complement store (counted for every word, an upper bound)."""
    return 16 + 4 + 24 + 8 + e_blocks * (112 if gibbs else 48)


PROFILE = ROOT / "profiles" / "lattice_kernel_batched_tapt_L10_R32_B256.md"


def load_traffic(source_hash):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel sources (lines "- source_sha256: ..." and "- dram_bytes_per_launch: ...")."""
    if not PROFILE.exists():
        return None
    kv = {}
    for line in PROFILE.read_text().splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256") != source_hash:
        return None
    try:
        return {"dram_bytes_per_launch": int(kv["dram_bytes_per_launch"])}
    except (KeyError, ValueError):
        return None


def source_hash():
    """sha256 of the lattice kernel's sources with comments and blank lines removed, so a
    comment edit does not invalidate the profile's counters."""
    import re
    h = hashlib.sha256()
    for name in ("pt_lattice.cuh", "pt_lattice.cu", "pt_device.cuh", "pt_layout.h"):
        text = (ROOT / "paper_2509_23043_gb300" / "csrc" / name).read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [ln.split("//", 1)[0].rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()


# ------------------------------------------------------------------------------ served stream
def served_stream(args, stream):
    """Poisson arrivals of EA +-J requests (L uniform over --serve-L), each run by TAPT in the
    continuous-batching server to within 0.1% of its reference lowest energy or the sweep
    budget; the same requests run one instance per launch with plain PT (no proposals).
    Reference energies: the best of --serve-ref-runs independent PT runs of
    --serve-ref-sweeps sweeps, each best configuration's energy recomputed on the host. Pools
    (PT runs of this library) and reference energies are made first and are not part of any
    time-to-solution; the pools' sweeps per request are reported beside it, and a second
    served run uses pools that cost about as many sweeps as plain PT's median time to the
    target. A third served run has a device-memory budget small enough to bind."""
    import instances as I
    import paper_2509_23043_gb300 as pt
    from paper_2509_23043_gb300 import serve as S
    g = np.random.default_rng(0x5E7E)
    Ls = [int(x) for x in args.serve_L.split(",")]
    R, P = 32, 256
    betas = I.geometric_betas(0.1, 3.0, R)
    prop = [1] * (R - 2) + [0, 0]
    n = args.serve_requests
    req_L = [int(g.choice(Ls)) for _ in range(n)]
    insts = [I.ea_instance(L, seed=0x5E5E, index=k) for k, L in enumerate(req_L)]
    ids = [10_000 + k for k in range(n)]
    t0 = time.perf_counter()
    pools = S.make_pools(insts, [betas] * n, ids, P, burnin=args.serve_pool_burnin,
                         gap=args.serve_pool_gap, stream=stream)
    pool_sweeps = args.serve_pool_burnin + args.serve_pool_gap * P
    eref = S.reference_energies(insts, [betas] * n, ids, sweeps=args.serve_ref_sweeps, chunk=2000,
                                runs=args.serve_ref_runs, verify=True, stream=stream)
    prep_s = time.perf_counter() - t0
    unit = np.cumsum(g.exponential(1.0, size=n))        # arrival pattern, scaled by the mean gap
    unit -= unit[0]
    mk = lambda k, a, pl=None: S.Request(ids[k], insts[k], betas, prop, pools[k] if pl is None else pl[k],
                                         eref[k], arrival=float(a))
    cfg = pt.Config(seed=0x7A972509, propose_every=10, propose_start=0, pool_size=P)
    slots = {L: 4 for L in Ls}
    footprint_all = sum(4 * S.footprint_bytes(L, R, P) for L in Ls)
    budget = int(args.serve_hbm_frac * footprint_all)
    gap_s, capacity = args.serve_gap_ms * 1e-3, None
    if args.serve_load > 0:
        # capacity: the completion rate of the TAPT server with every request submitted at
        # once (n / makespan, admission limited by slots and the device-memory budget); the
        # measured stream then arrives at serve_load x capacity
        cal = S.TaptServer(slots, betas, prop, cfg, hbm_budget=budget, tick_cycles=100,
                           stream=stream)
        done = cal.serve([mk(k, 0.0) for k in range(n)], budget_sweeps=args.serve_budget)
        capacity = n / max(r.finished for r in done)
        gap_s = 1.0 / (args.serve_load * capacity)
    arrivals = unit * gap_s
    srv = S.TaptServer(slots, betas, prop, cfg, hbm_budget=budget, tick_cycles=100, stream=stream)
    served = srv.serve([mk(k, arrivals[k]) for k in range(n)], budget_sweeps=args.serve_budget)
    cfg_pt = pt.Config(seed=0x7A972509, propose_every=0, pool_size=0)
    # the same server without proposals: separates the gain of batching from that of TAPT
    srv_pt = S.TaptServer(slots, betas, prop, cfg_pt, hbm_budget=budget, tick_cycles=100,
                          stream=stream)
    served_pt = srv_pt.serve([S.Request(ids[k], insts[k], betas, prop, None, eref[k],
                                        arrival=float(arrivals[k])) for k in range(n)],
                             budget_sweeps=args.serve_budget)
    alone = [S.run_alone(mk(k, 0.0), cfg_pt, budget_sweeps=args.serve_budget, tick_cycles=100,
                         stream=stream) for k in range(n)]
    alone_sum = S.summarize(alone)
    # pools that cost about as many sweeps per request as plain PT needs to reach the target
    # (its median over the solved requests): half burn-in, half captures
    med = max(2 * P, int(alone_sum.get("solved_p50_sweeps", 2 * P)))
    cheap_burn, cheap_gap = med // 2, max(1, (med // 2) // P)
    cheap = S.make_pools(insts, [betas] * n, ids, P, burnin=cheap_burn, gap=cheap_gap, seed=0x9002,
                         stream=stream)
    srv_c = S.TaptServer(slots, betas, prop, cfg, hbm_budget=budget, tick_cycles=100, stream=stream)
    served_c = srv_c.serve([mk(k, arrivals[k], cheap) for k in range(n)], budget_sweeps=args.serve_budget)
    # a device-memory budget that binds: every request submitted at once, a budget of the
    # footprint of four of the largest slots, so requests wait for memory with slots free
    tight = 4 * S.footprint_bytes(max(Ls), R, P)
    srv_m = S.TaptServer(slots, betas, prop, cfg, hbm_budget=tight, tick_cycles=100, stream=stream)
    served_m = srv_m.serve([mk(k, 0.0) for k in range(n)], budget_sweeps=args.serve_budget)
    s_tapt, s_cheap = S.summarize(served), S.summarize(served_c)
    for sm, ps in ((s_tapt, pool_sweeps), (s_cheap, cheap_burn + cheap_gap * P)):
        sm["pool_sweeps_per_request"] = ps
        if "p50_sweeps" in sm:
            sm["amortised_p50_sweeps"] = sm["p50_sweeps"] + ps
    s_mem = S.summarize(served_m)
    s_mem.update({"hbm_budget_bytes": tight, "peak_bytes_admitted": srv_m.peak_used,
                  "peak_requests_in_flight": srv_m.peak_active})
    return {"workload": f"{n} requests, L uniform in {{{args.serve_L}}}, R={R}, Poisson arrivals "
                        f"(mean gap {gap_s * 1e3:.2f} ms), target E_ref + 0.1%|E_ref| "
                        f"(E_ref: best of {args.serve_ref_runs} PT runs of {args.serve_ref_sweeps} "
                        f"sweeps, energies recomputed on the host), budget {args.serve_budget} sweeps "
                        f"(a request stopped by it counts as censored at the budget), pools P={P} from "
                        f"PT runs of {args.serve_pool_burnin} + {args.serve_pool_gap * P} sweeps "
                        f"(untimed; {prep_s:.1f} s with the reference runs)",
            "served_tapt": s_tapt,
            "served_tapt_pools_at_pt_cost": s_cheap,
            "served_tapt_memory_bound": s_mem,
            "served_plain_pt": S.summarize(served_pt),
            "plain_pt_one_instance_per_launch": alone_sum,
            "slots_per_L": 4, "hbm_budget_bytes": budget, "peak_bytes_admitted": srv.peak_used,
            "peak_requests_in_flight": srv.peak_active,
            "admission": "device memory modelled: every slot is allocated when the server is "
                         "built; the budget caps the summed footprint of the admitted requests",
            "capacity_per_s": capacity, "offered_per_s": 1.0 / gap_s,
            "load": (1.0 / gap_s) / capacity if capacity else None}


# ------------------------------------------------------------------------------ other workloads
def _time_ms(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(reps):
        fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def plain_pt_single(stream):
    """One EA instance, L=6, 16 slots (beta 0.2 -> 3.0), 10^4 sweeps of plain PT in one launch."""
    import instances as I
    import paper_2509_23043_gb300 as pt
    inst = I.ea_instance(6, index=0)
    betas = I.geometric_betas(0.2, 3.0, 16)
    ctx = pt.create_instances([inst], [betas], pt.Config(seed=0x7A972509), instance_ids=[0],
                              stream=stream.cuda_stream)
    ms = _time_ms(lambda: pt.run_cycles(ctx, 10_000), 3, stream)
    att = 16 * 216 * 10_000
    pt.destroy(ctx)
    return {"workload": "plain PT, 1 EA instance L=6, R=16, 10^4 sweeps in one launch",
            "ms": ms, "attempts_per_ns": att / (ms * 1e6)}


def engine_comparison(stream, B=256, L=10, R=32, P=64, cycles=100, reps=5):
    """The batched-TAPT workload (256 EA L=10, R=32 on 0.1 -> 3.0, proposals every 10 sweeps on
    30 slots), with Metropolis (the benchmark's rule) and Gibbs (the paper's rule), on both
    engines under one protocol: the bit-packed lattice engine (32 walkers per word), and the
    int8 graph engine, given the same lattices as general graphs (DSATUR finds their two
    colours). Pools of P from short PT runs of each engine (untimed); block sizes autotuned per
    engine; no L2 flush (the state lives in shared memory)."""
    import instances as I
    import paper_2509_23043_gb300 as pt
    lat = [I.ea_instance(L, index=k) for k in range(B)]
    gra = [I.Instance(i.n_spins, i.edge_i, i.edge_j, i.edge_J, None, None, 0) for i in lat]
    betas = [I.geometric_betas(0.1, 3.0, R)] * B
    prop = [[1] * (R - 2) + [0, 0]] * B
    ids = list(range(B))
    out = {}
    for rule, update in (("metropolis", pt.METROPOLIS), ("gibbs", pt.GIBBS)):
        for name, insts in (("bit_packed_lattice_engine", lat), ("int8_graph_engine", gra)):
            cfg = pt.Config(update=update, seed=0x7A972509, propose_every=10, propose_start=0,
                            pool_size=P)
            ctx = pt.create_instances(insts, betas, cfg, prop_enabled=prop, instance_ids=ids,
                                      stream=stream.cuda_stream)
            gen = pt.create_instances(insts, betas, pt.Config(update=update, seed=0x9001),
                                      instance_ids=[2_000_000 + i for i in ids],
                                      stream=stream.cuda_stream)
            pt.run_cycles(gen, 2000)
            for e in range(P):
                pt.run_cycles(gen, 2)
                pt.capture_proposals(ctx, gen, e)
            pt.destroy(gen)
            pt.autotune(ctx, probe_cycles=20)
            ms = _time_ms(lambda: pt.run_cycles(ctx, cycles), reps, stream)
            out[f"{rule}_{name}"] = {"engine": pt.info(ctx)["engine"],
                                     "threads_per_block": pt.info(ctx)["threads"],
                                     "ms_per_100_cycles": ms * 100 / cycles,
                                     "attempts_per_ns": B * R * L ** 3 * cycles / (ms * 1e6)}
            pt.destroy(ctx)
    return {"workload": f"{B} EA L={L}, R={R}, proposals every 10 from pools of {P}, "
                        f"{cycles} cycles per launch, autotuned block sizes, no L2 flush",
            "engines": out}


def ragged_batch(stream, n=4096, P=512, cycles=100, reps=5, cpu_pool=None, e2e_steps=5,
                 flush=None):
    """4096 EA instances, L uniform in {6..16} (even), R uniform in 24..48 on 0.1 -> 3.0,
    proposals every 10 sweeps from pools of 512 (PT runs of this library, untimed), block
    sizes autotuned per size class, cycles replayed from a CUDA graph: the largest configuration
    on one GPU. Beside its throughput: its ALU roofline (the algorithmic count of each size
    class, its plane blocks per word from a state sample of two members), an end-to-end rate
    through the public API (each step's pool window copied in from pinned host memory, the
    energies read back), and the oracle on the host cores on a sample of the same mix."""
    import torch
    import instances as I
    import paper_2509_23043_gb300 as pt
    g = np.random.default_rng(3)
    Ls = g.choice([6, 8, 10, 12, 14, 16], size=n)
    Rs = g.integers(24, 49, size=n)
    insts = [I.ea_instance(int(L), index=k) for k, L in enumerate(Ls)]
    betas = [I.geometric_betas(0.1, 3.0, int(R)) for R in Rs]
    props = [[1] * (int(R) - 2) + [0, 0] for R in Rs]
    ids = list(range(n))
    cfg = pt.Config(seed=0x7A972509, propose_every=10, propose_start=0, pool_size=P)
    t0 = time.perf_counter()
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=props, instance_ids=ids,
                              stream=stream.cuda_stream)
    gen = pt.create_instances(insts, betas, pt.Config(seed=0x9001),
                              instance_ids=[1_000_000 + i for i in ids], stream=stream.cuda_stream)
    pt.run_cycles(gen, 2000)
    for e in range(P):
        pt.run_cycles(gen, 4)
        pt.capture_proposals(ctx, gen, e)
    pt.destroy(gen)
    pt.autotune(ctx, probe_cycles=20)
    prep = time.perf_counter() - t0
    ms = _time_ms(lambda: pt.run_cycles_graph(ctx, cycles), reps, stream)
    att = int(sum(int(R) * int(L) ** 3 for L, R in zip(Ls, Rs))) * cycles
    groups = pt.group_info(ctx)
    value = att / (ms * 1e6)
    # roofline: the algorithmic ALU count of every word, by size class (L, walker blocks),
    # counted for the occupied lanes only (R/32 words per site), so padding lanes of a
    # partly filled walker block add no work
    cls = {}
    for k, (L, R) in enumerate(zip(Ls, Rs)):
        cls.setdefault((int(L), (int(R) + 31) // 32), []).append(k)
    ops = words = 0.0
    eb_w = 0.0
    for key, members in cls.items():
        eb = float(np.mean([plane_blocks_of(ctx, k, insts[k], "metropolis") for k in members[:2]]))
        w = sum(int(Ls[k]) ** 3 * int(Rs[k]) / 32.0 for k in members) * cycles
        ops += alu_ops_per_word(eb) * w
        words += w
        eb_w += eb * w
    peak = pt.calibrate_int(0)[0] / 1e12
    achieved = ops / (ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "lattice_kernel",
                "alu_ops_per_attempt": ops / att,
                "plane_blocks_per_word": eb_w / words,
                "peak_basis": "measured in this run by pt_calibrate_int (independent lop3.b32 on "
                              "every SM)",
                "note": "algorithmic count per size class over the occupied lanes, plane blocks "
                        "from two members each"}
    # end to end: each step's window of pool entries copied in (pinned host memory), energies out
    e2e = None
    if e2e_steps > 0:
        per_step = cycles // cfg.propose_every
        c, _ = pt.read_counters(ctx, 0)
        first = int(c[2]) % P
        need = min(P, per_step * e2e_steps)
        nws = [(int(L) ** 3 + 31) // 32 for L in Ls]
        slab = int(sum(int(R) * nw for R, nw in zip(Rs, nws)))
        host = torch.empty((need, slab), dtype=torch.int32, pin_memory=True)
        for j in range(need):                     # the entries the timed steps will use
            pt.read_proposals_packed(ctx, host[j].data_ptr(), (first + j) % P, 1)
        eout = torch.empty(sum(int(R) for R in Rs), dtype=torch.int32, device="cuda")
        ehost = torch.empty_like(eout, device="cpu").pin_memory()
        t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t_a.record(stream)
        for st in range(e2e_steps):
            if flush is not None:
                flush.zero_()
            for j in range(per_step):
                jj = (st * per_step + j) % need
                pt.load_proposals_packed(ctx, host[jj].data_ptr(), (first + st * per_step + j) % P, 1)
            pt.run_cycles_graph(ctx, cycles)
            pt.energies_device(ctx, eout.data_ptr())
            ehost.copy_(eout, non_blocking=True)
        t_b.record(stream)
        torch.cuda.synchronize()
        ms2 = t_a.elapsed_time(t_b) / e2e_steps
        e2e = {"value": att / (ms2 * 1e6), "unit": "attempts/ns",
               "h2d_bytes_per_step": per_step * slab * 4, "d2h_bytes_per_step": int(eout.numel()) * 4,
               "steps": e2e_steps,
               "note": "each step's pool window copied in from pinned host memory on the "
                       "launch stream before its cycles; L2 flushed between steps inside the "
                       "timed region"}
        del host
    pt.destroy(ctx)
    cpu = None
    if cpu_pool is not None:
        cpu = ragged_cpu_oracle(Ls[:16], Rs[:16], 40, cpu_pool)
    return {"workload": f"{n} EA instances, L in {{6..16}}, R in 24..48, proposals every 10 "
                        f"from pools of {P} (2000 + {4 * P} PT sweeps per instance, untimed), "
                        f"autotuned, {cycles} graph-replayed cycles per step",
            "value": value, "unit": "attempts/ns", "ms_per_step": ms, "attempts_per_ns": value,
            "size_classes": len(groups), "gpu_launches_per_step": len(groups),
            "threads_per_class": sorted({gr["threads"] for gr in groups}), "prep_s": round(prep, 1),
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu}


def ragged_cpu_oracle(Ls, Rs, sweeps, pool):
    """The oracle on the host cores on a sample of the ragged mix: the given (L, R) pairs, one
    process per instance, random pools of 64 per slot."""
    cores = min(os.cpu_count() or 1, len(Ls))
    jobs = [(int(L), int(R), k, sweeps, 0x7A972509, 0) for k, (L, R) in enumerate(zip(Ls, Rs))]
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    return {"value": sum(r[0] for r in res) / (wall * 1e9), "unit": "attempts/ns", "cores": cores,
            "kind": "oracle",
            "sample": f"{len(Ls)} instances of the ragged mix (L, R as the batch's first 16) x "
                      f"{sweeps} cycles each, one process per instance on {cores} host cores"}


def _mark_factored(ctx, mult, products, solved_at, sweeps):
    """Success of a factorization run (S4): some replica decodes to A * B = C with A, B > 1.
    Marks every instance k not yet solved whose state succeeds now with `sweeps`."""
    import paper_2509_23043_gb300 as pt
    wA = 1 << np.arange(mult.w)
    for k in np.nonzero(solved_at < 0)[0]:
        sp, _ = pt.read_state(ctx, int(k))
        A = (sp[:, mult.A] > 0) @ wA
        B = (sp[:, mult.B] > 0) @ wA
        if np.any((A * B == products[k]) & (A > 1) & (B > 1)):
            solved_at[k] = sweeps


def graph_alu_ops_per_attempt(mean_degree: float) -> float:
    """Algorithmic integer-ALU operations of one attempt of the graph engine (int8 spins,
    eight walkers of one site per thread, Gibbs or Metropolis): 2.5 for the three-input XORs
    of one Philox4x32-10 call shared by the eight walkers (20 / 8; its wide multiplies run on
    the FMA pipe; the second call, for the low halves of the uniforms, runs only at a tie and
    is not counted), mean_degree / 8 to decode the packed row entries (one per neighbour,
    shared by the eight walkers; the byte-sum multiply-adds run on the FMA pipe), and 7 per
    walker: extract its byte of the field sum, form the threshold index, compare the high
    halves, test for a tie, form and insert the new spin byte, and its energy term."""
    return 2.5 + mean_degree / 8.0 + 7.0


def _oracle_worker_factor(a):
    C, R, index, sweeps, seed = a
    sys.path.insert(0, str(ROOT))
    import instances as I
    import oracle as O
    inst = I.multiplier(8).instance(C)
    betas = I.geometric_betas(0.05, 5.0, R)
    P = 64
    o = O.Oracle(inst, betas, instance_id=index, prop_enabled=[1] * 23 + [0] * (R - 23), update=1,
                 propose_every=10, propose_start=0, seed=seed, pool_size=P)
    for r in range(R):
        o.load_pool(r, I.random_configs(inst.n_spins, P, index=r))
    t0 = time.perf_counter()
    o.run_cycles(sweeps)
    return R * int((inst.clamp == 0).sum()) * sweeps, time.perf_counter() - t0


def factorization(stream, sweeps_total, n=1000, R=32, P=512, burn=100_000, gap=25, chunk=1000,
                  cpu_pool=None):
    """The 8x8-bit multiplier (N = 200) with the product bits clamped to n products of two
    primes <= 255; R = 32 on 0.05 -> 5.0, proposals every 10 sweeps on the 23 hottest slots,
    Gibbs (the paper's rule) and Metropolis. Per-product pools: P configurations of each
    product's own clamped instance, captured every `gap` sweeps of one PT run after `burn`
    sweeps (untimed), shared by both rules. Success: some replica decodes to A*B = C with
    A, B > 1."""
    import instances as I
    import paper_2509_23043_gb300 as pt
    mult = I.multiplier(8)
    prods = I.draw_prime_products(n)
    betas = I.geometric_betas(0.05, 5.0, R)
    prop = [1] * 23 + [0] * (R - 23)
    insts = [mult.instance(C) for C, _, _ in prods]
    ctxs = {}
    for name, upd in (("gibbs", pt.GIBBS), ("metropolis", pt.METROPOLIS)):
        # colour classes of at most 32 free sites: one pass each of a 128-thread block
        cfg = pt.Config(update=upd, seed=0x7A972509, propose_every=10, propose_start=0,
                        pool_size=P, colour_cap=32)
        ctxs[name] = pt.create_instances(insts, [betas] * n, cfg, prop_enabled=[prop] * n,
                                         instance_ids=list(range(n)), stream=stream.cuda_stream)
    t0 = time.perf_counter()
    gen = pt.create_instances(insts, [betas] * n, pt.Config(update=pt.GIBBS, seed=0x9001, colour_cap=32),
                              instance_ids=[7_000_000 + k for k in range(n)],
                              stream=stream.cuda_stream)
    left = burn
    while left > 0:
        pt.run_cycles(gen, min(left, 10_000))
        left -= 10_000
    for e in range(P):
        pt.run_cycles(gen, gap)
        for ctx in ctxs.values():
            pt.capture_proposals(ctx, gen, e)
    pt.destroy(gen)
    stream.synchronize()
    prep = time.perf_counter() - t0
    att = n * R * int((insts[0].clamp == 0).sum())
    free = insts[0].clamp == 0
    deg = np.zeros(insts[0].n_spins)
    np.add.at(deg, insts[0].edge_i, 1)
    np.add.at(deg, insts[0].edge_j, 1)
    ops_att = graph_alu_ops_per_attempt(float(deg[free].mean()))
    peak = pt.calibrate_int(0)[0] / 1e12
    out = {"workload": f"{n} clamped 8x8-bit multipliers (N={mult.n_spins}), R={R} on "
                       f"0.05->5.0, proposals every 10 sweeps on 23 slots from per-product pools "
                       f"of {P} (a clamped PT run of {burn} + {P}x{gap} sweeps, untimed, "
                       f"{prep:.1f} s)"}
    for name, ctx in ctxs.items():
        solved_at = np.full(n, -1)
        done, t_gpu = 0, 0.0
        checkpoints = {}
        while done < sweeps_total:
            step = min(chunk, sweeps_total - done)
            s, e = _ev_pair()
            s.record(stream)
            pt.run_cycles(ctx, step)
            e.record(stream)
            e.synchronize()
            t_gpu += s.elapsed_time(e)
            done += step
            _mark_factored(ctx, mult, [C for C, _, _ in prods], solved_at, done)
            checkpoints[done] = int((solved_at >= 0).sum())
        pt.destroy(ctx)
        rate = att * done / (t_gpu * 1e6)
        out[name] = {"attempts_per_ns": rate,
                     "solved_of": n, "solved_after_sweeps": checkpoints,
                     "median_sweeps_to_solution": (float(np.median(solved_at[solved_at >= 0]))
                                                   if (solved_at >= 0).any() else None),
                     "roofline": {"bound": "alu", "achieved": rate * ops_att * 1e9 / 1e12,
                                  "peak": peak, "unit": "TOP/s",
                                  "frac": rate * ops_att * 1e9 / 1e12 / peak, "traffic": None,
                                  "kernel": "graph_kernel", "alu_ops_per_attempt": ops_att,
                                  "peak_basis": "measured in this run by pt_calibrate_int"}}
    if cpu_pool is not None:
        jobs = [(int(C), R, k, 20, 0x7A972509) for k, (C, _, _) in enumerate(prods[:16])]
        t0 = time.perf_counter()
        res = cpu_pool.map(_oracle_worker_factor, jobs)
        wall = time.perf_counter() - t0
        cores = min(os.cpu_count() or 1, len(jobs))
        out["cpu_baseline"] = {"value": sum(r[0] for r in res) / (wall * 1e9), "unit": "attempts/ns",
                               "cores": cores, "kind": "oracle",
                               "sample": f"{len(jobs)} of the clamped multipliers x 20 Gibbs cycles each "
                                         f"(random pools of 64), one process per instance on {cores} host cores"}
    return out


def _chain_bank(stream, src, betas, chains, captures, burn, gap, seed, id0):
    """A proposal bank from independent PT chains of this library: `chains` chains per source
    instance, each burned in for `burn` sweeps, then captured `captures` times `gap` sweeps
    apart. uint32 [captures * chains][len(src)][R * ceil(N/32)]; entry c * chains + j is
    capture c of chain j, so consecutive entries come from different chains."""
    import paper_2509_23043_gb300 as pt
    m, R = len(src), len(betas)
    nw = (src[0].n_spins + 31) // 32
    gi = [inst for inst in src for _ in range(chains)]
    ids = [id0 + i for i in range(len(gi))]
    gen = pt.create_instances(gi, [betas] * len(gi), pt.Config(update=pt.GIBBS, seed=seed),
                              instance_ids=ids, stream=stream.cuda_stream)
    dst = pt.create_instances(gi, [betas] * len(gi),
                              pt.Config(update=pt.GIBBS, seed=1, pool_size=captures),
                              instance_ids=ids, stream=stream.cuda_stream)
    left = burn
    while left > 0:
        pt.run_cycles(gen, min(left, 10_000))
        left -= 10_000
    for c in range(captures):
        pt.run_cycles(gen, gap)
        pt.capture_proposals(dst, gen, c)
    words = np.zeros((captures, len(gi) * R * nw), dtype=np.uint32)
    pt.read_proposals_packed(dst, words, 0, captures)
    pt.destroy(gen)
    pt.destroy(dst)
    return (words.reshape(captures, m, chains, R * nw).transpose(0, 2, 1, 3)
            .reshape(captures * chains, m, R * nw))


def factorization_tts(stream, w=8, n_products=32, runs=32, R=32, t_max=50000, check=1000,
                      chains=256, captures=4, burn=100_000, gap=250, n_prop=23,
                      modes=("plain_pt", "tapt_universal_bank", "tapt_instance_bank")):
    """Time to solution of Supplementary S5 on the w x w multiplier (2w-bit products of two
    primes below 2^w): every product is run `runs` times independently by plain PT and by
    TAPT, which proposes once per sweep on the n_prop hottest of R slots from a pre-generated
    bank (untimed). A bank holds captures of `chains` independent PT chains of this library:
    of each product's clamped instance (one bank per product), or of the universal
    (unclamped) circuit (one bank for all). The runs of a product share its bank, each
    starting at its own random entry. s(t_a) per product from its runs; TTS*_MCS = min over
    t_a of t_a * ceil(log 0.01 / log(1 - s(t_a))), converted to seconds with the measured
    device time per run and sweep. Reported: medians over the products."""
    import instances as I
    import paper_2509_23043_gb300 as pt
    from paper_2509_23043_gb300 import tts as TT
    mult = I.multiplier(w)
    prods = I.draw_prime_products(n_products, max_factor=(1 << w) - 1, seed=0x7755)
    betas = I.geometric_betas(0.05, 5.0, R)
    prop = [1] * n_prop + [0] * (R - n_prop)
    P = chains * captures
    insts = [mult.instance(C) for C, _, _ in prods for _ in range(runs)]
    ids = [1000 * k + j for k in range(n_products) for j in range(runs)]
    n = len(insts)
    checks = list(range(check // 10, check, check // 10)) + list(range(check, t_max + 1, check))
    t0 = time.perf_counter()
    banks = {}
    if "tapt_universal_bank" in modes:
        banks["tapt_universal_bank"] = _chain_bank(stream, [mult.instance(None)], betas, chains,
                                                   captures, burn, gap, 0x9004, 6_000_000)
    if "tapt_instance_bank" in modes:
        banks["tapt_instance_bank"] = _chain_bank(stream, [mult.instance(C) for C, _, _ in prods],
                                                  betas, chains, captures, burn, gap, 0x9005,
                                                  6_100_000)
    prep = time.perf_counter() - t0
    start = np.random.default_rng(0x57A7).integers(0, P, size=n)      # each run's first entry
    entry = (np.arange(P)[:, None] + start[None, :]) % P
    out = {}
    for name in modes:
        kw = {} if name == "plain_pt" else dict(propose_every=1, propose_start=0, pool_size=P)
        cfg = pt.Config(update=pt.GIBBS, seed=0x7A97, **kw)
        ctx = pt.create_instances(insts, [betas] * n, cfg, prop_enabled=[prop] * n,
                                  instance_ids=ids, stream=stream.cuda_stream)
        if kw:
            bank = banks[name]
            owner = np.arange(n) // runs if bank.shape[1] > 1 else np.zeros(n, dtype=np.int64)
            words = np.ascontiguousarray(bank[entry, owner[None, :], :]).reshape(P, -1)
            pt.load_proposals_packed(ctx, words, 0, P)
            stream.synchronize()
            del words
        solved_at = np.full(n, -1)
        t_ms, done = 0.0, 0
        for t in checks:
            a_, b_ = _ev_pair()
            a_.record(stream)
            pt.run_cycles(ctx, t - done)
            b_.record(stream)
            b_.synchronize()
            t_ms += a_.elapsed_time(b_)
            done = t
            _mark_factored(ctx, mult, [prods[k // runs][0] for k in range(n)], solved_at, t)
        pt.destroy(ctx)
        per_sweep_s = t_ms * 1e-3 / (n * t_max)          # device time per run and sweep
        best = np.array([TT.optimal_tts(checks, TT.success_curve(
            solved_at[k * runs:(k + 1) * runs], checks)) for k in range(n_products)])
        tts_mcs = best[:, 0]
        finite = np.isfinite(tts_mcs)
        med = float(np.median(tts_mcs))
        out[name] = {"median_tts_sweeps": med if np.isfinite(med) else None,
                     "median_tts_s": med * per_sweep_s if np.isfinite(med) else None,
                     "median_best_run_length": float(np.median(best[finite, 1])) if finite.any() else None,
                     "products_with_finite_tts": int(finite.sum()),
                     "runs_solved": int((solved_at >= 0).sum()),
                     "us_per_run_sweep": round(per_sweep_s * 1e6, 4),
                     "device_ms": round(t_ms, 1)}
    return {"workload": f"{n_products} products of two primes < 2^{w} on the {w}x{w} multiplier "
                        f"(N={mult.n_spins}), {runs} independent runs each, R={R} on 0.05->5.0, "
                        f"Gibbs, {t_max} sweeps checked every {check // 10} up to {check}, then "
                        f"every {check}; TAPT proposes every sweep on {n_prop} slots from banks of {P}: "
                        f"{chains} independent PT chains x {captures} captures {gap} sweeps apart "
                        f"after {burn} (untimed, {prep:.1f} s for both kinds)",
            "target_success": TT.P_TARGET, "modes": out}


def tts_scaling(stream, ws=(8, 9, 10), n_products=32, runs=23,
                modes=("plain_pt", "tapt_universal_bank", "tapt_instance_bank"), growth=2):
    """The scaling fit of Fig. 5 (S5): median TTS* at product sizes n = 2w, then
    TTS(n) = A exp(k n) by least squares on log TTS, for plain PT and both TAPT banks, in
    sweeps and in seconds. Run lengths grow with n (5e4 * growth^(w-8) sweeps). 32 x 23 runs
    keep every size in one wave of CTAs (760 fit at w = 10, limited by shared memory)."""
    from paper_2509_23043_gb300 import tts as TT
    per = {}
    for w in ws:
        f = growth ** (w - 8)
        per[2 * w] = factorization_tts(stream, w=w, n_products=n_products, runs=runs,
                                       t_max=50_000 * f, check=1000 * f, modes=modes)
    modes = list(next(iter(per.values()))["modes"])
    fits = {}
    for m in modes:
        fits[m] = {}
        for unit in ("sweeps", "s"):
            med = [per[n]["modes"][m][f"median_tts_{unit}"] for n in per]
            fit = TT.fit_exponent(list(per), [np.inf if v is None else v for v in med])
            fits[m][f"k_{unit}"] = None if fit is None else fit[1]
            fits[m][f"median_tts_{unit}"] = dict(zip(per, med))
    return {"workload": f"product bits n in {sorted(per)}, {n_products} products x {runs} runs "
                        f"each, as the time-to-solution workload",
            "fit": "log TTS = log A + k n, least squares over the per-size medians",
            "modes": fits,
            "per_size": {n: {m: {k: v for k, v in d.items() if k != "device_ms"}
                             for m, d in per[n]["modes"].items()} for n in per}}


def large_lattice(stream, n=152, L=20, R=64, P=16, cycles=20, reps=3):
    """Lattices too large for shared memory: n EA instances of L = 20 (N = 8000) with R = 64
    (two walker blocks: 128 KB of spins and 128 KB of neighbour table per instance, kept in
    global memory and L2), Metropolis, proposals every 10 cycles from random pools of P,
    autotuned, with the same ALU roofline count as the main workload."""
    import paper_2509_23043_gb300 as pt
    import instances as I
    insts = [I.ea_instance(L, index=50_000 + k) for k in range(n)]
    betas = I.geometric_betas(0.1, 3.0, R)
    cfg = pt.Config(seed=0x1A46E, propose_every=10, propose_start=0, pool_size=P)
    ctx = pt.create_instances(insts, [betas] * n, cfg, prop_enabled=[[1] * (R - 2) + [0, 0]] * n,
                              instance_ids=list(range(n)), stream=stream.cuda_stream)
    nw = (L ** 3 + 31) // 32
    rng = np.random.default_rng(0x1A46E)
    for e0 in range(0, P, 4):
        words = rng.integers(0, 2 ** 32, size=(4, n, R, nw), dtype=np.uint64).astype(np.uint32)
        pt.load_proposals_packed(ctx, words, e0, 4)
        stream.synchronize()
    pt.autotune(ctx, probe_cycles=5)
    pt.run_cycles(ctx, 40)
    stream.synchronize()
    best = 1e30
    for _ in range(reps):
        s0, e0 = _ev_pair()
        s0.record(stream)
        pt.run_cycles(ctx, cycles)
        e0.record(stream)
        e0.synchronize()
        best = min(best, s0.elapsed_time(e0))
    rate = n * R * L ** 3 * cycles / (best * 1e6)
    e_blocks = plane_blocks_of(ctx, 0, insts[0], "metropolis")
    ops = alu_ops_per_word(e_blocks) / 32
    peak = pt.calibrate_int(0)[0] / 1e12
    g = pt.group_info(ctx)[0]
    pt.destroy(ctx)
    return {"workload": f"{n} EA +-J instances, L={L} (N={L ** 3}), R={R}, Metropolis, proposals every 10 "
                        f"cycles from random pools of {P}, spins and neighbour table in global memory "
                        f"(the instance does not fit shared memory), autotuned, {cycles} cycles per launch",
            "attempts_per_ns": rate, "ms_per_launch": best, "threads_per_block": g["threads"],
            "shared_memory_per_block": g["smem"],
            "roofline": {"bound": "alu", "achieved": rate * ops * 1e9 / 1e12, "peak": peak, "unit": "TOP/s",
                         "frac": rate * ops * 1e9 / 1e12 / peak, "traffic": None, "kernel": "lattice_kernel (GSP)",
                         "alu_ops_per_attempt": ops, "plane_blocks_per_word": e_blocks,
                         "peak_basis": "measured in this run by pt_calibrate_int"}}


def ladder_workload(stream, n=64, R=32, iterations=6, sweeps=2000):
    """Ladder optimisation for uniform swap acceptance on the EA L=10 family (a shared
    ladder, R=32 on 0.1 -> 3.0, starting geometric): swap acceptance per pair before and
    after, from the library's own exchange statistics."""
    import instances as I
    from paper_2509_23043_gb300 import ladder as LD
    insts = [I.ea_instance(10, seed=0x1ADD, index=k) for k in range(n)]
    b0 = I.geometric_betas(0.1, 3.0, R)
    t0 = time.perf_counter()
    b, hist = LD.optimise_ladder(insts, b0, iterations=iterations, sweeps=sweeps,
                                 stream=stream.cuda_stream)
    _, last = LD.optimise_ladder(insts, b, iterations=1, sweeps=sweeps, seed=0x2ADD,
                                 stream=stream.cuda_stream)
    wall = time.perf_counter() - t0
    a0, a1 = hist[0]["acceptance"], last[0]["acceptance"]
    return {"workload": f"{n} EA L=10 instances, R={R} on 0.1->3.0, {iterations} rounds of "
                        f"{sweeps} PT sweeps, then one check round",
            "acceptance_geometric": {"min": float(a0.min()), "max": float(a0.max()),
                                     "mean": float(a0.mean())},
            "acceptance_optimised": {"min": float(a1.min()), "max": float(a1.max()),
                                     "mean": float(a1.mean())},
            "betas": [round(float(x), 4) for x in b], "wall_s": round(wall, 2)}


def context_ablation(stream, n=64, L=10, R=32, sweeps=3000, chunk=500):
    """Supplementary S3-style comparison on n EA L=10 instances, R=32 on 0.1 -> 3.0: plain PT,
    pool proposals (PT-run pools, as in the main workload) and contextual proposals keeping
    50 / 25 / 12.5 % of the spins (2 refill sweeps), every 10 sweeps from sweep 100 on the 30
    hottest slots. Reported: mean residual energy per spin of the best slot against a long
    PT reference (2e5 sweeps, untimed), at checkpoints, and the device time of each run."""
    import instances as I
    import paper_2509_23043_gb300 as pt
    from paper_2509_23043_gb300 import serve as SV
    insts = [I.ea_instance(L, seed=0xC0DE, index=k) for k in range(n)]
    betas = I.geometric_betas(0.1, 3.0, R)
    prop = [1] * (R - 2) + [0, 0]
    ids = list(range(n))
    eref = np.array(SV.reference_energies(insts, [betas] * n, ids, sweeps=200_000, chunk=5000,
                                          stream=stream.cuda_stream))
    pools = SV.make_pools(insts, [betas] * n, ids, 256, burnin=20_000, gap=40,
                          stream=stream.cuda_stream)
    N = L ** 3
    modes = {"plain_pt": dict(),
             "pool": dict(propose_every=10, propose_start=100, pool_size=256),
             "context_50": dict(propose_every=10, propose_start=100, proposal_source=1,
                                context_log2=1, context_sweeps=2),
             "context_25": dict(propose_every=10, propose_start=100, proposal_source=1,
                                context_log2=2, context_sweeps=2),
             "context_12": dict(propose_every=10, propose_start=100, proposal_source=1,
                                context_log2=3, context_sweeps=2)}
    out = {}
    for name, kw in modes.items():
        ctx = pt.create_instances(insts, [betas] * n, pt.Config(seed=0xAB1A, **kw),
                                  prop_enabled=[prop] * n, instance_ids=ids,
                                  stream=stream.cuda_stream)
        if kw.get("pool_size"):
            for k in range(n):
                pt.load_proposals_inst_packed(ctx, k, pools[k])
        best = np.full(n, 10 ** 9)
        curve, t_ms, done = {}, 0.0, 0
        while done < sweeps:
            s, e = _ev_pair()
            s.record(stream)
            pt.run_cycles(ctx, chunk)
            e.record(stream)
            e.synchronize()
            t_ms += s.elapsed_time(e)
            done += chunk
            best = np.minimum(best, np.array([x.min() for x in pt.energies(ctx)]))
            curve[done] = float(np.mean((best - eref) / N))
        pt.destroy(ctx)
        out[name] = {"residual_per_spin": curve, "device_ms": round(t_ms, 2)}
    return {"workload": f"{n} EA L={L} instances, R={R} on 0.1->3.0, {sweeps} sweeps, proposals "
                        f"every 10 from sweep 100 on {R - 2} slots; reference: best of 2e5 PT "
                        f"sweeps", "modes": out}


def isingformer_workload(stream, B=1024, reps=5):
    """IsingFormer inference at the paper's spin-glass and factorization shape (d_model 256,
    4 heads, 5 layers, FFN 1024; Methods and Supplementary S6) over the 8x8-bit multiplier's
    N = 200 spins in the factorization order {C}{carry}{multiplier}{B}{A}, seeded bfloat16
    weights. Scoring: log q(x | beta) of B configurations in one teacher-forced pass (the
    Hastings factor of an MH move with a learned q). Sampling: B configurations drawn one
    position after another, the product and carry-in bits given as the clamped prefix
    (Supplementary S6), replayed from a CUDA graph. Tensor roofline of the matrix products
    (bfloat16 inputs, FP32 accumulation) against the measured bfloat16 peak."""
    import torch
    import instances as I
    from paper_2509_23043_gb300.former import Former
    mult = I.multiplier(8)
    N = mult.n_spins
    shp = I.FormerShape(n_spins=N)
    W, packed = I.former_weights(shp)
    m = Former(shp, packed, stream=stream.cuda_stream)
    g = np.random.default_rng(0xF0F0)
    X = torch.from_numpy(np.where(g.random((B, N)) < 0.5, 1, -1).astype(np.int8)).cuda()
    beta = torch.from_numpy(I.geometric_betas(0.05, 5.0, 32)[g.integers(0, 23, B)].astype(np.float32)).cuda()
    ms = _time_ms(lambda: m.score(X, beta), reps, stream)
    gemm = m.score_gemm_flops(B)
    attn = shp.n_layers * shp.n_heads * B * (N * (N + 1) / 2) * 64 * 4.0
    peak_tf = _measured_peak("bf16_tflops")
    # sampling with the product and carry-in bits of a product as the prefix
    inst = mult.instance(251 * 241)
    npre = int((inst.clamp != 0).sum())
    assert np.all(inst.clamp[:npre] != 0), "the clamped bits lead the factorization order"
    pre = torch.from_numpy(np.tile(inst.clamp[:npre], (B, 1)).astype(np.int8)).cuda()
    out = torch.empty((B, N), dtype=torch.int8, device="cuda")
    lq = torch.empty(B, dtype=torch.float32, device="cuda")
    m.sample(beta, 1, 0, prefix=pre, out=out, logq=lq)        # direct launches + capture
    ms_s = _time_ms(lambda: m.sample(beta, 2, 0, prefix=pre, out=out, logq=lq), reps, stream)
    # sampling is latency-bound at this B (N sequential steps of small products): the same
    # call for 8 times as many configurations
    Bl = 8 * B
    beta_l = beta.repeat(8)
    pre_l = pre.repeat(8, 1)
    out_l = torch.empty((Bl, N), dtype=torch.int8, device="cuda")
    lq_l = torch.empty(Bl, dtype=torch.float32, device="cuda")
    m.sample(beta_l, 1, 0, prefix=pre_l, out=out_l, logq=lq_l)
    ms_sl = _time_ms(lambda: m.sample(beta_l, 2, 0, prefix=pre_l, out=out_l, logq=lq_l), 2, stream)
    del out_l, lq_l
    # end to end: configurations in from pinned host memory, log q out, every call
    hx = X.cpu().pin_memory()
    hq = torch.empty(B, dtype=torch.float32).pin_memory()
    dx = torch.empty_like(X)

    def e2e_call():
        dx.copy_(hx, non_blocking=True)
        hq.copy_(m.score(dx, beta), non_blocking=True)
    ms_e = _time_ms(e2e_call, reps, stream)
    out_d = {"workload": f"IsingFormer d_model 256, 4 heads, 5 layers, FFN 1024, seeded bfloat16 "
                         f"weights, N = {N} (8x8 multiplier), B = {B} configurations per call",
             "score": {"configs_per_s": B / (ms * 1e-3), "ms_per_call": ms,
                       "roofline": {"bound": "tensor", "achieved": gemm / (ms * 1e-3) / 1e12,
                                    "peak": peak_tf, "unit": "TFLOP/s",
                                    "frac": gemm / (ms * 1e-3) / 1e12 / peak_tf if peak_tf else None,
                                    "traffic": None, "kernel": "the scoring pass (this library's "
                                    "tcgen05 kernels for the first FFN map with bias and GELU "
                                    "fused and for the whole causal attention: scores, softmax "
                                    "and P V; the other projections on cuBLASLt; norms, "
                                    "embedding and head in this library's kernels)",
                                    "flops_per_call": gemm, "attention_flops_per_call": attn,
                                    "note": "projection FLOPs over the whole pass's time; the "
                                            "attention's causal products (Q K^T and P V below "
                                            "the diagonal) are reported beside them"}},
             "sample": {"configs_per_s": B / (ms_s * 1e-3), "ms_per_call": ms_s, "prefix": npre,
                        "gpu_launches_per_call": "one CUDA graph of N steps",
                        f"configs_per_s_B{8 * B}": Bl / (ms_sl * 1e-3), f"ms_per_call_B{8 * B}": ms_sl,
                        "roofline": sample_roofline(shp, Bl, ms_sl, elem_bytes=2)},
             "e2e": {"value": B / (ms_e * 1e-3), "unit": "configs/s", "h2d_bytes_per_step": B * N,
                     "d2h_bytes_per_step": B * 4}}
    out_d["score"]["hbm_view"] = score_hbm_view(shp, B, ms)
    # the same pass with every projection on cuBLASLt (proj_mode 1) and with every suitable
    # projection on the tcgen05 kernels (proj_mode 2)
    for mode in (1, 2):
        alt = Former(shp, packed, stream=stream.cuda_stream, proj_mode=mode)
        out_d["score"][f"ms_per_call_proj_mode_{mode}"] = _time_ms(lambda: alt.score(X, beta), reps, stream)
        alt.check()
        del alt
    m.check()
    # the oracle on the host cores (numpy float64, BLAS threads): a few configurations
    from oracle import former as F
    t0 = time.perf_counter()
    F.score(W, shp, X[:8].cpu().numpy(), beta[:8].cpu().numpy().astype(np.float64))
    dt = time.perf_counter() - t0
    out_d["cpu_baseline"] = {"value": 8 / dt, "unit": "configs/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": "8 configurations scored by the float64 "
                             "numpy oracle (BLAS threads on the host cores)"}
    del m
    return out_d


def score_hbm_view(shp, B, ms):
    """The scoring pass against the copy bandwidth: the bytes its kernels hand to one another
    through HBM, M = B N rows. Per layer: the first layer norm reads the FP32 residual stream
    and writes bfloat16 (6 M d; folded into the embedding at layer 0), QKV reads it and writes
    3 d columns (8 M d), the fused attention reads QKV and writes O (8 M d), the output map reads
    O and reads and writes the stream (10 M d), the second layer norm (6 M d), the first FFN
    map (2 M d + 2 M F), the second (2 M F + 8 M d): 48 M d + 4 M F. Plus the embedding's write
    of the stream and the head's read of it."""
    N, d, F, L = shp.n_spins, shp.d_model, shp.d_ff, shp.n_layers
    M = B * N
    nbytes = L * (48.0 * M * d + 4.0 * M * F) - (4.0 * M * d if L else 0.0) + 8.0 * M * d
    peak = _measured_peak("hbm_gbs")
    ach = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if peak else None, "bytes_per_call": nbytes,
            "note": "activation bytes between the pass's kernels over the whole pass's time"}


def sample_roofline(shp, B, ms, elem_bytes=2):
    """HBM roofline of autoregressive sampling: at step t every layer reads the cached key and
    value rows 0..t of each configuration (2 d values per row, bfloat16 in the default mode)
    and appends row t, so a call moves L B 2d e (N(N+1)/2 + N) bytes of cache; the weights (a
    few MB, resident in L2) and the per-step activations (B rows) are left out."""
    N, d, L = shp.n_spins, shp.d_model, shp.n_layers
    nbytes = L * B * 2 * d * float(elem_bytes) * (N * (N + 1) / 2 + N)
    peak = _measured_peak("hbm_gbs")
    ach = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if peak else None, "traffic": None, "configs_per_call": B,
            "kernel": "the sampling call (one CUDA graph of N steps; the attention-step kernel "
                      "streams the bfloat16 key/value cache)", "bytes_per_call": nbytes,
            "note": "key/value cache bytes over the whole call's time"}


def _measured_peak(key):
    p = ROOT / "MEASURED_PEAKS.json"
    try:
        return float(json.loads(p.read_text())[key])
    except (OSError, KeyError, ValueError):
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0}.get(key)


def _ev_pair():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ------------------------------------------------------------------------------ CPU oracle
def _oracle_worker(a):
    L, R, index, sweeps, seed, update = a
    sys.path.insert(0, str(ROOT))
    import instances as I
    import oracle as O
    inst = I.ea_instance(L, index=index)
    betas = I.geometric_betas(0.1, 3.0, R)
    P = 64
    o = O.Oracle(inst, betas, instance_id=index, prop_enabled=[1] * (R - 2) + [0, 0],
                 propose_every=10, propose_start=0, seed=seed, pool_size=P, update=update)
    for r in range(R):
        o.load_pool(r, I.random_configs(inst.n_spins, P, index=r))
    t0 = time.perf_counter()
    o.run_cycles(sweeps)
    return R * inst.n_spins * sweeps, time.perf_counter() - t0


def cpu_oracle(args, n_inst, sweeps, pool=None):
    import multiprocessing as mp
    cores = min(os.cpu_count() or 1, n_inst)
    jobs = [(args.L, args.R, k, sweeps, 0x7A972509, update_rule(args)) for k in range(n_inst)]
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    if own:
        pool.close()
        pool.join()
    attempts = sum(r[0] for r in res)
    return {"value": attempts / (wall * 1e9), "unit": "attempts/ns", "cores": cores,
            "kind": "oracle", "wall_s": wall,
            "sample": f"{n_inst} instances of the workload (L={args.L}, R={args.R}) x {sweeps} "
                      f"cycles each, one process per instance on {cores} host cores"}


# ------------------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    n_inst, sweeps = args.cpu_sample_instances, max(10, args.cpu_sample_sweeps // 2)
    cores = min(os.cpu_count() or 1, n_inst)
    pool = mp.get_context("spawn").Pool(cores)
    for _ in range(args.warmup):
        cpu_oracle(args, cores, 2, pool)
    # each step's sample is sized so that the K timed steps take about two minutes in all
    probe = cpu_oracle(args, n_inst, 2, pool)
    per_cycle_s = max(probe["wall_s"] / 2, 1e-6)
    sweeps = int(max(2, min(sweeps, 120.0 / (max(args.steps, 1) * per_cycle_s))))
    tot_att, tot_t = 0, 0.0
    for _ in range(args.steps):
        r = cpu_oracle(args, n_inst, sweeps, pool)
        tot_att += r["value"] * r["wall_s"] * 1e9
        tot_t += r["wall_s"]
    pool.close()
    pool.join()
    v = tot_att / (tot_t * 1e9)
    sample = (f"each step: {n_inst} instances of the workload (L={args.L}, R={args.R}) x "
              f"{sweeps} cycles, one process per instance on {cores} host cores")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "attempts/ns",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i8",
        "dtype_detail": "int8 spins, int32 energies, f64 acceptance (the oracle)",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "global_batch": args.instances,
                   "timed": "a bounded sample of the workload per step, on the host cores "
                            "(see cpu_baseline.sample)"},
        "cpu_baseline": {"value": v, "unit": "attempts/ns", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "attempts/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------ profiler cases
def profile_case(kind):
    """Small cases for ncu captures (the commands are in profiles/). lattice, lattice-gibbs:
    the benchmark workload (256 EA L=10, R=32, proposals every 10 from sweep 100) with random
    pools of 1024 entries (1 GB, larger than L2), one launch at creation then four of 100
    cycles. graph: 1000 clamped 8x8 multipliers, Gibbs, colour classes of at most 32 free
    sites, pools of 16, one launch at creation then three of 1000 cycles. former: three IsingFormer scoring passes over 1024
    configurations of N = 200. former-sample: one IsingFormer sampling call of 1024
    configurations of N = 200 with the product and carry-in bits as the prefix (direct
    launches: 200 steps; a 1 GB bfloat16 key/value cache)."""
    import torch
    import instances as I
    import paper_2509_23043_gb300 as pt
    torch.cuda.set_device(0)
    rng = np.random.default_rng(1)
    if kind.startswith("lattice"):
        class A:
            L, R, threads = 10, 32, 0
        n, P, L, R = 256, 1024, 10, 32
        insts, betas, prop, ids = workload(A, 0, n)
        cfg = pt.Config(update=1 if kind == "lattice-gibbs" else 0, sweeps_per_cycle=1, propose_every=10,
                        propose_start=100, pool_size=P, seed=0x7A972509)
        ctx = pt.create_instances(insts, betas, cfg, prop_enabled=prop, instance_ids=ids)
        nw = (L ** 3 + 31) // 32
        for e0 in range(0, P, 64):
            words = rng.integers(0, 2 ** 32, size=(64, n, R, nw), dtype=np.uint64).astype(np.uint32)
            pt.load_proposals_packed(ctx, words, e0, 64)
            torch.cuda.synchronize()
        for _ in range(4):
            pt.run_cycles(ctx, 100)
        out = pt.energies(ctx)[:4]
    elif kind == "graph":
        nB, R, P = 1000, 32, 16
        mult = I.multiplier(8)
        insts = [mult.instance(C) for C, _, _ in I.draw_prime_products(nB)]
        betas = I.geometric_betas(0.05, 5.0, R)
        cfg = pt.Config(update=pt.GIBBS, seed=0x7A972509, propose_every=10, propose_start=0, pool_size=P,
                        colour_cap=32)
        ctx = pt.create_instances(insts, [betas] * nB, cfg, prop_enabled=[[1] * 23 + [0] * (R - 23)] * nB,
                                  instance_ids=list(range(nB)))
        nw = (mult.n_spins + 31) // 32
        words = rng.integers(0, 2 ** 32, size=(P, nB, R, nw), dtype=np.uint64).astype(np.uint32)
        pt.load_proposals_packed(ctx, words, 0, P)
        torch.cuda.synchronize()
        for _ in range(3):
            pt.run_cycles(ctx, 1000)
        out = pt.energies(ctx)[:4]
    elif kind == "former-sample":
        from paper_2509_23043_gb300.former import Former
        mult = I.multiplier(8)
        shp = I.FormerShape(n_spins=mult.n_spins)
        _, packed = I.former_weights(shp)
        m = Former(shp, packed)
        inst = mult.instance(251 * 241)
        npre = int((inst.clamp != 0).sum())
        pre = torch.from_numpy(np.tile(inst.clamp[:npre], (1024, 1)).astype(np.int8)).cuda()
        beta = torch.full((1024,), 1.0, dtype=torch.float32, device="cuda")
        S, lq = m.sample(beta, 1, 0, prefix=pre)
        m.check()
        out = lq[:4].cpu().numpy()
    else:
        from paper_2509_23043_gb300.former import Former
        shp = I.FormerShape(n_spins=200)
        _, packed = I.former_weights(shp)
        m = Former(shp, packed)
        X = torch.from_numpy(np.where(rng.random((1024, 200)) < 0.5, 1, -1).astype(np.int8)).cuda()
        beta = torch.full((1024,), 1.0, dtype=torch.float32, device="cuda")
        for _ in range(3):
            lq = m.score(X, beta)
        out = lq[:4].cpu().numpy()
    torch.cuda.synchronize()
    print("profile case", kind, "ok", out)


# ------------------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args.profile_case)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the CPU baseline's process pool starts before the first GPU call
    cpu_pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mp
        cpu_pool = mp.get_context("spawn").Pool(min(os.cpu_count() or 1, args.cpu_sample_instances))
    import torch
    import paper_2509_23043_gb300 as pt
    from paper_2509_23043_gb300 import shard
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    B = args.instances
    first = shard.weak_shard(rank, world, B).start
    insts, betas, prop, ids = workload(args, first, B)
    cfg = make_config(args, args.pool_size)
    ctx = pt.create_instances(insts, betas, cfg, prop_enabled=prop, instance_ids=ids,
                              stream=stream.cuda_stream)
    t_pool = time.perf_counter()
    build_pools(args, insts, betas, prop, ids, ctx)
    torch.cuda.synchronize()
    t_pool = time.perf_counter() - t_pool
    spc = args.sweeps_per_step
    attempts_per_step = B * args.R * args.L ** 3 * spc

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step():
        pt.run_cycles(ctx, spc)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e_blocks = expected_plane_blocks(ctx, args) if rank == 0 else 0.0

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.wait_first()
        t_start = time.monotonic()
        for k in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps (untimed)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk.mark(t_start, time.monotonic())
    if dist:
        dist.barrier()
    ms = shard.job_ms(sum(a.elapsed_time(b) for a, b in ev), dist, device="cuda")
    ms_step = ms / args.steps
    value = shard.job_rate(attempts_per_step * args.steps, world, ms)

    # ---------------- end to end through the public API: host pool window in, energies out
    e2e = None
    if not args.no_e2e:
        nw = (args.L ** 3 + 31) // 32
        slab = B * args.R * nw
        per_step_entries = spc // cfg.propose_every
        assert args.pool_size >= 2 * per_step_entries, "pipelined windows need two disjoint windows"
        # pinned host copy of the device pool, so reloading a window changes nothing
        host_pool = torch.empty((args.pool_size, slab), dtype=torch.int32, pin_memory=True)
        pt.read_proposals_packed(ctx, host_pool.data_ptr(), 0, args.pool_size)
        eout = torch.empty(B * args.R, dtype=torch.int32, device="cuda")
        ehost = torch.empty(B * args.R, dtype=torch.int32, pin_memory=True)
        c, _ = pt.read_counters(ctx, 0)
        # Pipelined: step k's window is copied on a second stream while step k-1 runs (the
        # windows are disjoint pool entries); step k waits for its copy. Every copy, kernel,
        # L2 flush and energies read-back lies between the two timing events.
        copy = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(args.steps)]

        def load_window(k):
            first_e = (int(c[2]) + k * per_step_entries) % args.pool_size
            left = per_step_entries
            pt.set_stream(ctx, copy.cuda_stream)
            while left > 0:
                take = min(left, args.pool_size - first_e)
                pt.load_proposals_packed(ctx, host_pool.data_ptr() + first_e * slab * 4, first_e, take)
                left -= take
                first_e = 0
            pt.set_stream(ctx, stream.cuda_stream)
            ev_in[k].record(copy)

        t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t_a.record(stream)
        copy.wait_stream(stream)
        load_window(0)
        for k in range(args.steps):
            flush.zero_()
            stream.wait_event(ev_in[k])
            if k + 1 < args.steps:
                load_window(k + 1)
            step()
            pt.energies_device(ctx, eout.data_ptr())
            ehost.copy_(eout, non_blocking=True)
        t_b.record(stream)
        torch.cuda.synchronize()
        ms2 = shard.job_ms(t_a.elapsed_time(t_b), dist, device="cuda")
        e2e = {"value": shard.job_rate(attempts_per_step * args.steps, world, ms2), "unit": "attempts/ns",
               "h2d_bytes_per_step": per_step_entries * slab * 4,
               "d2h_bytes_per_step": B * args.R * 4,
               "note": "the next step's pool window is copied while the current step runs; "
                       "L2 flushes inside the timed region"}

    # ---------------- roofline of the dominant kernel (the fused cycle kernel = the whole step)
    words_per_step = B * args.L ** 3 * ((args.R + 31) // 32) * spc
    ops = alu_ops_per_word(e_blocks, args.update == "gibbs") * words_per_step
    achieved = ops / (ms_step * 1e-3) / 1e12
    nominal = SM_COUNT * ALU_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    measured, _ = pt.calibrate_int(0)
    peak = measured / 1e12
    # the committed capture is of the Metropolis instantiation
    tr = load_traffic(source_hash()) if args.update == "metropolis" else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s",
                "frac": achieved / peak,
                "traffic": (tr["dram_bytes_per_launch"] if tr else None),
                "kernel": "lattice_kernel", "alu_ops_per_attempt": alu_ops_per_word(e_blocks, args.update == "gibbs") / 32,
                "plane_blocks_per_word": e_blocks,
                "peak_basis": "measured in this run by pt_calibrate_int (independent lop3.b32 "
                              "on every SM); nominal 152 SMs x 64 ALU lanes x 2070 MHz = "
                              f"{nominal:.2f} TOP/s"}
    smem_peak, _ = pt.calibrate_smem()
    smem_achieved = smem_bytes_per_word(e_blocks, args.update == "gibbs") * words_per_step / (ms_step * 1e-3)
    roofline["smem"] = {"achieved_gbs": smem_achieved / 1e9, "peak_gbs": smem_peak / 1e9,
                        "frac": smem_achieved / smem_peak,
                        "bytes_per_attempt": smem_bytes_per_word(e_blocks, args.update == "gibbs") / 32,
                        "peak_basis": "measured in this run by pt_calibrate_smem (conflict-free "
                                      "16-byte shared loads on every SM)"}

    serving = None
    ragged = None
    if not args.no_serve and rank == 0:
        serving = served_stream(args, stream.cuda_stream)
    others = None
    if not args.no_configs and rank == 0:
        wl = set(args.workloads.split(","))
        others = {}
        if "plain" in wl:
            others["plain_pt_single"] = plain_pt_single(stream)
        if "engines" in wl:
            others["engine_comparison"] = engine_comparison(stream)
        if "ragged" in wl:
            ragged = ragged_batch(stream, cpu_pool=cpu_pool, flush=flush)
        if "factor" in wl:
            others["factorization"] = factorization(stream, args.factor_sweeps,
                                                    P=args.factor_pool_size,
                                                    burn=args.factor_pool_burnin,
                                                    gap=args.factor_pool_gap, cpu_pool=cpu_pool)
        if "ladder" in wl:
            others["ladder"] = ladder_workload(stream)
        if "large" in wl:
            others["large_lattice"] = large_lattice(stream)
        if "tts" in wl:
            others["factorization_tts"] = factorization_tts(stream)
        if "tts_scaling" in wl:
            others["tts_scaling"] = tts_scaling(stream)
        if "tts_scaling_pt" in wl:
            # plain PT alone over the paper's full range of product sizes, n = 16 .. 24
            others["tts_scaling_pt"] = tts_scaling(stream, ws=(8, 9, 10, 11, 12), runs=19,
                                                   modes=("plain_pt",), growth=3)
        if "context" in wl:
            others["context_ablation"] = context_ablation(stream)
        if "former" in wl:
            others["isingformer"] = isingformer_workload(stream)

    cpu = None
    if cpu_pool is not None:
        cpu = cpu_oracle(args, args.cpu_sample_instances, args.cpu_sample_sweeps, cpu_pool)
        cpu_pool.close()
        cpu_pool.join()
        cpu.pop("wall_s", None)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "attempts/ns", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32",
            "dtype_detail": "u32 bit-packed spins (32 walkers per word), int32 energies, f64 acceptance",
            "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "global_batch": B * world, "l2": "flushed between timed steps",
                       "pool_generation_s": round(t_pool, 2),
                       "pool": f"PT runs of this library: {args.pool_burnin} burn-in sweeps, "
                               f"then one capture every {args.pool_gap} sweeps (untimed)",
                       "threads_per_block": pt.info(ctx)["threads"]},
            "other_workloads": others, "serving": serving,
            "ragged_batch_4096": ragged,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps, "clocks": clk.summary(),
        }), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
