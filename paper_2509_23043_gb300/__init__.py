"""GB300-native parallel tempering with global proposals (TAPT, arXiv 2509.23043).

A thin ctypes binding of libpt.so (include/pt.h). Each function below has the name of the
C entry point without its ``pt_`` prefix and only marshals arguments: every step of the
method runs in the library's CUDA kernels. There is no CPU fallback: if libpt.so is
missing or cannot be loaded the first call raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from pathlib import Path
from typing import Sequence

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "libpt.so"

PT_OK, PT_EINVAL, PT_ENOMEM, PT_ECUDA, PT_ETIMEOUT, PT_ESTATE, PT_ENOTSUP = range(7)
_STATUS = {0: "PT_OK", 1: "PT_EINVAL", 2: "PT_ENOMEM", 3: "PT_ECUDA", 4: "PT_ETIMEOUT",
           5: "PT_ESTATE", 6: "PT_ENOTSUP"}
METROPOLIS, GIBBS = 0, 1
DELTA_E_ONLY, ALWAYS_ACCEPT, INDEPENDENT_MH = 0, 1, 2     # proposal rules
POOL, CONTEXT = 0, 1                   # proposal sources


class PTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(C.Structure):
    _fields_ = [("instance_id", C.c_uint32), ("n_spins", C.c_int32), ("lattice_L", C.c_int32),
                ("n_edges", C.c_int32), ("edge_i", C.c_void_p), ("edge_j", C.c_void_p),
                ("edge_J", C.c_void_p), ("h", C.c_void_p), ("clamp", C.c_void_p),
                ("n_replicas", C.c_int32), ("beta", C.c_void_p), ("prop_enabled", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("update", C.c_int32), ("sweeps_per_cycle", C.c_int32),
                ("propose_every", C.c_int32), ("propose_start", C.c_int32),
                ("propose_stop", C.c_int32), ("pool_size", C.c_int32), ("seed", C.c_uint64),
                ("threads_per_block", C.c_int32), ("proposal_rule", C.c_int32),
                ("proposal_source", C.c_int32), ("context_log2", C.c_int32),
                ("context_sweeps", C.c_int32), ("colour_cap", C.c_int32)]


EXPORTS = ["pt_create_instances", "pt_load_proposals", "pt_load_proposals_packed",
           "pt_read_proposals_packed", "pt_load_proposals_inst_packed",
           "pt_capture_proposals", "pt_sweep", "pt_global_propose", "pt_exchange",
           "pt_run_cycles", "pt_energies", "pt_energies_device", "pt_read_state",
           "pt_read_state_noalloc",
           "pt_read_walkers", "pt_write_state", "pt_read_counters", "pt_read_stats", "pt_info",
           "pt_group_info", "pt_autotune", "pt_load_proposal_law", "pt_run_cycles_graph", "pt_set_instance",
           "pt_set_active", "pt_set_stream", "pt_calibrate_int", "pt_calibrate_smem", "pt_destroy",
           "pt_last_error"]

_lib = None


def lib():
    """Load libpt.so (raises if it is absent: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2509_23043_gb300.build` (needs nvcc)")
    L = C.CDLL(str(LIB_PATH))
    vp, i32, i64p = C.c_void_p, C.c_int32, C.c_void_p
    sig = {
        "pt_create_instances": [C.POINTER(C.c_void_p), C.POINTER(_Desc), i32, C.POINTER(_Config), vp],
        "pt_load_proposals": [vp, i32, i32, vp, i32, i32],
        "pt_load_proposals_packed": [vp, vp, i32, i32],
        "pt_read_proposals_packed": [vp, vp, i32, i32],
        "pt_load_proposals_inst_packed": [vp, i32, vp, i32, i32],
        "pt_load_proposal_law": [vp, i32, i32, vp],
        "pt_capture_proposals": [vp, vp, i32],
        "pt_sweep": [vp, i32], "pt_global_propose": [vp], "pt_exchange": [vp],
        "pt_run_cycles": [vp, i32], "pt_energies": [vp, vp], "pt_energies_device": [vp, vp],
        "pt_read_state": [vp, i32, vp, vp], "pt_read_state_noalloc": [vp, i32, vp, vp],
        "pt_read_walkers": [vp, i32, vp],
        "pt_write_state": [vp, i32, vp, vp, i64p, vp], "pt_read_counters": [vp, i32, i64p, vp],
        "pt_read_stats": [vp, i32, vp, vp, vp, vp], "pt_info": [vp, i32, vp],
        "pt_group_info": [vp, i32, vp], "pt_autotune": [vp, i32, vp],
        "pt_run_cycles_graph": [vp, i32], "pt_set_instance": [vp, i32, C.POINTER(_Desc)],
        "pt_set_active": [vp, i32, i32],
        "pt_set_stream": [vp, vp], "pt_destroy": [vp],
        "pt_calibrate_int": [i32, vp, vp],
        "pt_calibrate_smem": [vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.pt_last_error.argtypes = []
    L.pt_last_error.restype = C.c_char_p
    _lib = L
    return L


def last_error() -> str:
    return lib().pt_last_error().decode()


def _check(status: int):
    if status != PT_OK:
        raise PTError(status, last_error())


def _arr(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _inst(ctx, inst: int) -> int:
    if not 0 <= inst < len(ctx.R):
        raise PTError(PT_EINVAL, f"instance {inst} out of range [0, {len(ctx.R)})")
    return inst


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


@dataclass
class Config:
    update: int = METROPOLIS
    sweeps_per_cycle: int = 1
    propose_every: int = 0
    propose_start: int = 0
    propose_stop: int = 0
    pool_size: int = 0
    seed: int = 0
    threads_per_block: int = 0
    proposal_rule: int = DELTA_E_ONLY
    proposal_source: int = POOL
    context_log2: int = 1
    context_sweeps: int = 1
    colour_cap: int = 0

    def _c(self) -> _Config:
        return _Config(self.update, self.sweeps_per_cycle, self.propose_every,
                       self.propose_start, self.propose_stop, self.pool_size,
                       self.seed & 0xFFFFFFFFFFFFFFFF, self.threads_per_block,
                       self.proposal_rule, self.proposal_source, self.context_log2,
                       self.context_sweeps, self.colour_cap)


class Context:
    """A pt_ctx handle; released by destroy() or when garbage collected."""

    def __init__(self, handle: int, R: list[int], N: list[int]):
        self.handle = C.c_void_p(handle)
        self.R = R
        self.N = N

    @property
    def n(self) -> int:
        return len(self.R)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.pt_destroy(self.handle)
            self.handle = None


def _desc(inst, beta, prop, iid, keep):
    b = _arr(beta, np.float64)
    ei, ej, eJ = _arr(inst.edge_i, np.int32), _arr(inst.edge_j, np.int32), _arr(inst.edge_J, np.int32)
    h = _arr(getattr(inst, "h", None), np.int32)
    cl = _arr(getattr(inst, "clamp", None), np.int8)
    pe = None if prop is None else _arr(prop, np.uint8)
    keep += [b, ei, ej, eJ, h, cl, pe]
    return _Desc(int(iid) & 0xFFFFFFFF, int(inst.n_spins), int(getattr(inst, "lattice_L", 0)),
                 len(ei), _ptr(ei), _ptr(ej), _ptr(eJ), _ptr(h), _ptr(cl), len(b), _ptr(b), _ptr(pe))


def create_instances(instances: Sequence, betas: Sequence, config: Config,
                     prop_enabled: Sequence | None = None, instance_ids: Sequence[int] | None = None,
                     stream=None) -> Context:
    """pt_create_instances. `instances[k]` has n_spins, edge_i, edge_j, edge_J, h, clamp and
    lattice_L; `betas[k]` is its ascending ladder; `prop_enabled[k]` its R_prop flags."""
    n = len(instances)
    keep = []
    descs = (_Desc * n)()
    for k, inst in enumerate(instances):
        b = _arr(betas[k], np.float64)
        ei, ej, eJ = _arr(inst.edge_i, np.int32), _arr(inst.edge_j, np.int32), _arr(inst.edge_J, np.int32)
        h = _arr(getattr(inst, "h", None), np.int32)
        cl = _arr(getattr(inst, "clamp", None), np.int8)
        pe = None if prop_enabled is None or prop_enabled[k] is None else _arr(prop_enabled[k], np.uint8)
        keep += [b, ei, ej, eJ, h, cl, pe]
        iid = k if instance_ids is None else int(instance_ids[k])
        descs[k] = _Desc(iid & 0xFFFFFFFF, int(inst.n_spins), int(getattr(inst, "lattice_L", 0)),
                         len(ei), _ptr(ei), _ptr(ej), _ptr(eJ), _ptr(h), _ptr(cl), len(b),
                         _ptr(b), _ptr(pe))
    cfg = config._c()
    out = C.c_void_p()
    s = stream if stream is not None else _default_stream()
    _check(lib().pt_create_instances(C.byref(out), descs, n, C.byref(cfg), C.c_void_p(s)))
    return Context(out.value, [len(betas[k]) for k in range(n)],
                   [int(i.n_spins) for i in instances])


def load_proposals(ctx: Context, inst: int, replica: int, spins, first: int = 0):
    s = _arr(spins, np.int8)
    _check(lib().pt_load_proposals(ctx.handle, inst, replica, _ptr(s), s.shape[0], first))


def load_proposal_law(ctx: Context, inst: int, replica: int, p_plus):
    """pt_load_proposal_law: P(spin i = +1) per site of the law slot `replica`'s pool entries are
    drawn from (proposal_rule 2, the independent Metropolis-Hastings move)."""
    _inst(ctx, inst)
    p = np.ascontiguousarray(p_plus, dtype=np.float64)
    if p.shape != (ctx.N[inst],):
        raise ValueError(f"p_plus must have shape ({ctx.N[inst]},)")
    _check(lib().pt_load_proposal_law(ctx.handle, inst, replica, _ptr(p)))


def load_proposals_packed(ctx: Context, words, first: int, count: int):
    """words: uint32 array (host, ideally pinned) [count][instance][slot][ceil(N/32)]."""
    w = words if isinstance(words, int) else None
    if w is None:
        arr = _arr(words, np.uint32)
        _check(lib().pt_load_proposals_packed(ctx.handle, _ptr(arr), first, count))
    else:
        _check(lib().pt_load_proposals_packed(ctx.handle, C.c_void_p(w), first, count))


def load_proposals_inst_packed(ctx: Context, inst: int, words, first: int = 0):
    """words: uint32 [count][R][ceil(N/32)] bit strings for instance `inst`."""
    _inst(ctx, inst)
    w = _arr(words, np.uint32)
    _check(lib().pt_load_proposals_inst_packed(ctx.handle, inst, _ptr(w), first, w.shape[0]))


def read_proposals_packed(ctx: Context, words, first: int, count: int):
    """words: a writable host buffer address (int) or a uint32 numpy array."""
    if isinstance(words, int):
        _check(lib().pt_read_proposals_packed(ctx.handle, C.c_void_p(words), first, count))
    else:
        if not (words.dtype == np.uint32 and words.flags.c_contiguous):
            raise ValueError("words must be a C-contiguous uint32 array")
        _check(lib().pt_read_proposals_packed(ctx.handle, _ptr(words), first, count))


def capture_proposals(dst: Context, src: Context, entry: int):
    _check(lib().pt_capture_proposals(dst.handle, src.handle, entry))


def sweep(ctx: Context, n_sweeps: int):
    _check(lib().pt_sweep(ctx.handle, n_sweeps))


def global_propose(ctx: Context):
    _check(lib().pt_global_propose(ctx.handle))


def exchange(ctx: Context):
    _check(lib().pt_exchange(ctx.handle))


def run_cycles(ctx: Context, n_cycles: int):
    _check(lib().pt_run_cycles(ctx.handle, n_cycles))


def energies(ctx: Context) -> list[np.ndarray]:
    out = np.zeros(sum(ctx.R), dtype=np.int32)
    _check(lib().pt_energies(ctx.handle, _ptr(out)))
    offs = np.cumsum([0] + ctx.R)
    return [out[offs[k]:offs[k + 1]] for k in range(ctx.n)]


def energies_device(ctx: Context, dev_ptr: int):
    _check(lib().pt_energies_device(ctx.handle, C.c_void_p(dev_ptr)))


def read_state(ctx: Context, inst: int):
    _inst(ctx, inst)
    R, N = ctx.R[inst], ctx.N[inst]
    s = np.zeros((R, N), dtype=np.int8)
    E = np.zeros(R, dtype=np.int32)
    _check(lib().pt_read_state(ctx.handle, inst, _ptr(s), _ptr(E)))
    return s, E


def read_state_noalloc(ctx: Context, inst: int):
    """pt_read_state_noalloc: as read_state, through the library's fixed device buffer."""
    _inst(ctx, inst)
    R, N = ctx.R[inst], ctx.N[inst]
    s = np.zeros((R, N), dtype=np.int8)
    E = np.zeros(R, dtype=np.int32)
    _check(lib().pt_read_state_noalloc(ctx.handle, inst, _ptr(s), _ptr(E)))
    return s, E


def read_walkers(ctx: Context, inst: int) -> np.ndarray:
    _inst(ctx, inst)
    w = np.zeros(ctx.R[inst], dtype=np.int32)
    _check(lib().pt_read_walkers(ctx.handle, inst, _ptr(w)))
    return w


def write_state(ctx: Context, inst: int, spins, walker, counters, cursors=None):
    s, w = _arr(spins, np.int8), _arr(walker, np.int32)
    c, cu = _arr(counters, np.int64), _arr(cursors, np.int32)
    _check(lib().pt_write_state(ctx.handle, inst, _ptr(s), _ptr(w), _ptr(c), _ptr(cu)))


def read_counters(ctx: Context, inst: int):
    _inst(ctx, inst)
    c = np.zeros(3, dtype=np.int64)
    cu = np.zeros(ctx.R[inst], dtype=np.int32)
    _check(lib().pt_read_counters(ctx.handle, inst, _ptr(c), _ptr(cu)))
    return c, cu


def read_stats(ctx: Context, inst: int):
    _inst(ctx, inst)
    R = ctx.R[inst]
    sa, st = np.zeros(max(R - 1, 1), np.int64), np.zeros(max(R - 1, 1), np.int64)
    pa, pt_ = np.zeros(R, np.int64), np.zeros(R, np.int64)
    _check(lib().pt_read_stats(ctx.handle, inst, _ptr(sa), _ptr(st), _ptr(pa), _ptr(pt_)))
    return sa[:R - 1], st[:R - 1], pa, pt_


def info(ctx: Context, inst: int = -1) -> dict:
    v = np.zeros(6, dtype=np.int32)
    _check(lib().pt_info(ctx.handle, inst, _ptr(v)))
    return {"n": int(v[0]), "engine": "lattice" if v[1] == 0 else "graph",
            "threads": int(v[2]), "smem": int(v[3]), "R": int(v[4]), "N": int(v[5])}


def group_info(ctx: Context) -> list[dict]:
    v = np.zeros(4, dtype=np.int32)
    _check(lib().pt_group_info(ctx.handle, -1, _ptr(v)))
    out = []
    for g in range(int(v[0])):
        _check(lib().pt_group_info(ctx.handle, g, _ptr(v)))
        out.append({"members": int(v[0]), "threads": int(v[1]), "smem": int(v[2]), "first": int(v[3])})
    return out


def autotune(ctx: Context, probe_cycles: int = 20) -> list[int]:
    n = len(group_info(ctx))
    t = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().pt_autotune(ctx.handle, probe_cycles, _ptr(t)))
    return [int(x) for x in t[:n]]


def run_cycles_graph(ctx: Context, n_cycles: int):
    _check(lib().pt_run_cycles_graph(ctx.handle, n_cycles))


def set_instance(ctx: Context, inst: int, instance, beta, prop_enabled=None, instance_id: int = 0):
    _inst(ctx, inst)
    keep = []
    d = _desc(instance, beta, prop_enabled, instance_id, keep)
    _check(lib().pt_set_instance(ctx.handle, inst, C.byref(d)))


def set_active(ctx: Context, inst: int, active: bool):
    _inst(ctx, inst)
    _check(lib().pt_set_active(ctx.handle, inst, 1 if active else 0))


def set_stream(ctx: Context, stream):
    _check(lib().pt_set_stream(ctx.handle, C.c_void_p(stream)))


def calibrate_int(kind: int = 0) -> tuple[float, float]:
    """pt_calibrate_int: (operations per second, best launch ms) of independent lop3 (kind 0)
    or multiply-add (kind 1) operations on the current device."""
    v, ms = C.c_double(0.0), C.c_double(0.0)
    _check(lib().pt_calibrate_int(kind, C.byref(v), C.byref(ms)))
    return v.value, ms.value


def calibrate_smem() -> tuple[float, float]:
    """pt_calibrate_smem: (shared-memory bytes loaded per second, best launch ms) on the
    current device."""
    v, ms = C.c_double(0.0), C.c_double(0.0)
    _check(lib().pt_calibrate_smem(C.byref(v), C.byref(ms)))
    return v.value, ms.value


def destroy(ctx: Context):
    if ctx.handle is not None and ctx.handle.value:
        _check(lib().pt_destroy(ctx.handle))
        ctx.handle = None
