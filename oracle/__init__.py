"""ctypes binding of the plain C oracle (pt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the
benchmark's CPU-baseline leg. The CUDA product path never imports this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pt_oracle.c"
_OUT = _HERE / "_build" / "liboracle.so"
# -ffp-contract=off: the thresholds and acceptance tests are evaluated exactly as written.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> Path:
    _OUT.parent.mkdir(exist_ok=True)
    if force or not _OUT.exists() or _OUT.stat().st_mtime < max(
            _SRC.stat().st_mtime, (_HERE / "pt_oracle.h").stat().st_mtime):
        tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(["gcc", *CFLAGS, str(_SRC), "-o", str(tmp), "-lm"], check=True)
        os.replace(tmp, _OUT)
    return _OUT


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(str(build()))
        P = C.POINTER
        L.or_philox.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.or_metropolis_threshold.argtypes = [C.c_double, C.c_int32]
        L.or_metropolis_threshold.restype = C.c_uint32
        L.or_gibbs_threshold.argtypes = [C.c_double, C.c_int32]
        L.or_gibbs_threshold.restype = C.c_uint32
        L.or_accept.argtypes = [C.c_double, C.c_uint32]
        L.or_accept.restype = C.c_int
        L.or_energy.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]
        L.or_energy.restype = C.c_int64
        L.or_create.argtypes = [C.c_uint32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                C.c_int32, C.c_int32, C.c_uint64, C.c_int32, C.c_int32,
                                C.c_int32, C.c_int32, C.c_int32]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_load_pool.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32]
        L.or_load_pool.restype = C.c_int
        L.or_load_law.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.or_load_law.restype = C.c_int
        for f in ("or_sweeps", "or_run_cycles"):
            getattr(L, f).argtypes = [C.c_void_p, C.c_int32]
        for f in ("or_propose", "or_exchange"):
            getattr(L, f).argtypes = [C.c_void_p]
        L.or_read.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_write.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_counters.argtypes = [C.c_void_p, C.c_void_p]
        L.or_set_counters.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_cursors.argtypes = [C.c_void_p, C.c_void_p]
        L.or_stats.argtypes = [C.c_void_p] + [C.c_void_p] * 4
        L.or_colouring.argtypes = [C.c_void_p, C.c_void_p]
        L.or_colouring.restype = C.c_int32
        L.or_cap_colours.argtypes = [C.c_void_p, C.c_int32]
        L.or_cap_colours.restype = C.c_int32
        L.or_bitplane.argtypes = [C.c_void_p]
        L.or_bitplane.restype = C.c_int32
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def metropolis_threshold(beta: float, dE: int) -> int:
    return int(lib().or_metropolis_threshold(beta, dE))


def gibbs_threshold(beta: float, I: int) -> int:
    return int(lib().or_gibbs_threshold(beta, I))


def accept(x: float, u: int) -> bool:
    return bool(lib().or_accept(x, u))


def energy(inst, spins) -> int:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    ei = np.ascontiguousarray(inst.edge_i, dtype=np.int32)
    ej = np.ascontiguousarray(inst.edge_j, dtype=np.int32)
    eJ = np.ascontiguousarray(inst.edge_J, dtype=np.int32)
    h = None if inst.h is None else np.ascontiguousarray(inst.h, dtype=np.int32)
    return int(lib().or_energy(inst.n_spins, len(ei), _ptr(ei), _ptr(ej), _ptr(eJ), _ptr(h),
                               _ptr(s)))


class Oracle:
    """One instance run by the oracle (Algorithm 1 restated sequentially)."""

    def __init__(self, inst, betas, *, instance_id: int = 0, prop_enabled=None,
                 update: int = 0, sweeps_per_cycle: int = 1, propose_every: int = 0,
                 propose_start: int = 0, propose_stop: int = 0, seed: int = 0,
                 pool_size: int = 0, proposal_rule: int = 0, proposal_source: int = 0,
                 context_log2: int = 1, context_sweeps: int = 1, colour_cap: int = 0):
        self.inst = inst
        self.N = int(inst.n_spins)
        self.R = len(betas)
        self._keep = [np.ascontiguousarray(inst.edge_i, dtype=np.int32),
                      np.ascontiguousarray(inst.edge_j, dtype=np.int32),
                      np.ascontiguousarray(inst.edge_J, dtype=np.int32),
                      None if inst.h is None else np.ascontiguousarray(inst.h, dtype=np.int32),
                      None if inst.clamp is None else np.ascontiguousarray(inst.clamp, dtype=np.int8),
                      np.ascontiguousarray(betas, dtype=np.float64),
                      None if prop_enabled is None else np.ascontiguousarray(prop_enabled, dtype=np.uint8)]
        ei, ej, eJ, h, cl, b, pe = self._keep
        self.h = lib().or_create(instance_id, self.N, int(inst.lattice_L), len(ei), _ptr(ei),
                                 _ptr(ej), _ptr(eJ), _ptr(h), _ptr(cl), self.R, _ptr(b),
                                 _ptr(pe), update, sweeps_per_cycle, propose_every,
                                 propose_start, propose_stop, seed & 0xFFFFFFFFFFFFFFFF,
                                 pool_size, proposal_rule, proposal_source, context_log2,
                                 context_sweeps)
        if not self.h:
            raise ValueError("oracle rejected the instance")
        if colour_cap > 0:
            lib().or_cap_colours(self.h, colour_cap)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def load_pool(self, r: int, spins, first: int = 0):
        s = np.ascontiguousarray(spins, dtype=np.int8)
        if lib().or_load_pool(self.h, r, _ptr(s), s.shape[0], first):
            raise ValueError("bad pool load")

    def load_law(self, r: int, p_plus):
        """Proposal law of slot r (proposal_rule 2): P(spin i = +1) per site."""
        p = np.ascontiguousarray(p_plus, dtype=np.float64)
        if lib().or_load_law(self.h, r, _ptr(p)):
            raise ValueError("bad proposal law")

    def sweeps(self, n: int):
        lib().or_sweeps(self.h, n)

    def propose(self):
        lib().or_propose(self.h)

    def exchange(self):
        lib().or_exchange(self.h)

    def run_cycles(self, n: int):
        lib().or_run_cycles(self.h, n)

    def read(self):
        s = np.zeros((self.R, self.N), dtype=np.int8)
        E = np.zeros(self.R, dtype=np.int32)
        w = np.zeros(self.R, dtype=np.int32)
        lib().or_read(self.h, _ptr(s), _ptr(E), _ptr(w))
        return s, E, w

    def write(self, spins, walker=None):
        s = np.ascontiguousarray(spins, dtype=np.int8)
        w = None if walker is None else np.ascontiguousarray(walker, dtype=np.int32)
        lib().or_write(self.h, _ptr(s), _ptr(w))

    def counters(self):
        c = np.zeros(3, dtype=np.int64)
        lib().or_counters(self.h, _ptr(c))
        return c

    def cursors(self):
        c = np.zeros(self.R, dtype=np.int32)
        lib().or_cursors(self.h, _ptr(c))
        return c

    def set_counters(self, counters, cursors=None):
        c = np.ascontiguousarray(counters, dtype=np.int64)
        cu = None if cursors is None else np.ascontiguousarray(cursors, dtype=np.int32)
        lib().or_set_counters(self.h, _ptr(c), _ptr(cu))

    def stats(self):
        R = self.R
        sa, st = np.zeros(max(R - 1, 1), np.int64), np.zeros(max(R - 1, 1), np.int64)
        pa, pt = np.zeros(R, np.int64), np.zeros(R, np.int64)
        lib().or_stats(self.h, _ptr(sa), _ptr(st), _ptr(pa), _ptr(pt))
        return sa[:R - 1], st[:R - 1], pa, pt

    def colouring(self):
        c = np.zeros(self.N, dtype=np.int32)
        n = lib().or_colouring(self.h, _ptr(c))
        return c, int(n)

    @property
    def bitplane(self) -> bool:
        return bool(lib().or_bitplane(self.h))
