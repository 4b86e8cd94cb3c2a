"""Seeded synthetic inputs for parallel tempering (PT) and its transformer-augmented
variant (TAPT).

This module builds problem instances and inputs only. It holds none of the method's
arithmetic: no update rule, no acceptance rule, no random stream that the method draws.
Both the CUDA library and the CPU oracle take what it produces as plain arrays.

Contents
- 3D Edwards-Anderson +-J spin glasses on a periodic L^3 lattice. These stand in for the
  D-Wave instances of the paper (Methods, "Benchmark instances"), which are not available.
- The invertible-multiplier Ising encoding used for factorization (Supplementary S4):
  AND gates and full adders, with the paper's J and h for each gate.
- Random 8-bit prime pairs, geometric inverse-temperature ladders, random proposal pools.

Conventions: spin m in {-1,+1}, logical 0 -> -1 and 1 -> +1 (Supplementary S4).
Energy E(m) = -sum_{i<j} J_ij m_i m_j - sum_i h_i m_i (Supplementary S4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 0x7A972509


def _rng(*keys: int) -> np.random.Generator:
    """A numpy generator keyed by a tuple of integers (no link to the method's streams)."""
    return np.random.default_rng(np.random.SeedSequence([int(k) & 0xFFFFFFFF for k in keys]))


@dataclass
class Instance:
    """One Ising instance as plain arrays (the energy-function input of Algorithm 1).

    edge_i, edge_j, edge_J: undirected couplings, one row per edge (parallel edges allowed).
    h: local fields or None. clamp: per-spin 0 (free) or +-1 (clamped), or None.
    lattice_L > 0 marks a periodic L^3 lattice whose edges are in canonical order
    (for site n = x + L*(y + L*z): its +x, +y, +z bonds, in that order).
    """
    n_spins: int
    edge_i: np.ndarray
    edge_j: np.ndarray
    edge_J: np.ndarray
    h: np.ndarray | None = None
    clamp: np.ndarray | None = None
    lattice_L: int = 0
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------------------
# 3D Edwards-Anderson +-J lattice (stand-in for the paper's D-Wave instances, Methods)
# ----------------------------------------------------------------------------------------

def ea_edges(L: int) -> tuple[np.ndarray, np.ndarray]:
    """Canonical bond list of the periodic L^3 lattice: 3 forward bonds per site."""
    if L < 2:
        raise ValueError("L must be >= 2")
    n = np.arange(L ** 3, dtype=np.int64)
    x, y, z = n % L, (n // L) % L, n // (L * L)
    nx = ((x + 1) % L) + L * (y + L * z)
    ny = x + L * (((y + 1) % L) + L * z)
    nz = x + L * (y + L * ((z + 1) % L))
    ei = np.repeat(n, 3)
    ej = np.stack([nx, ny, nz], axis=1).reshape(-1)
    return ei.astype(np.int32), ej.astype(np.int32)


def ea_instance(L: int, seed: int = MASTER_SEED, index: int = 0, p_neg: float = 0.5,
                ferro: bool = False) -> Instance:
    """Periodic 3D EA spin glass, J = -1 with probability p_neg else +1, no field."""
    ei, ej = ea_edges(L)
    if ferro:
        J = np.ones(ei.shape[0], dtype=np.int32)
    else:
        u = _rng(seed, 0xEA, L, index).random(ei.shape[0])
        J = np.where(u < p_neg, -1, 1).astype(np.int32)
    return Instance(L ** 3, ei, ej, J, None, None, L, {"kind": "ea", "L": L, "index": index})


def geometric_betas(b_min: float, b_max: float, R: int) -> np.ndarray:
    """Geometric ladder beta_k = b_min (b_max/b_min)^(k/(R-1)), ascending (hot -> cold)."""
    if R == 1:
        return np.array([b_min], dtype=np.float64)
    k = np.arange(R, dtype=np.float64)
    return b_min * (b_max / b_min) ** (k / (R - 1))


# ----------------------------------------------------------------------------------------
# Invertible multiplier (Supplementary S4): AND gates + full adders
# ----------------------------------------------------------------------------------------

# Gate parameters as printed in Supplementary S4 (upper triangle of J, and h).
AND_J = {(0, 1): -1, (0, 2): 2, (1, 2): 2}           # spins (A, B, C)
AND_H = (1, 1, -2)
FA_J = {(0, 1): -1, (0, 2): -1, (0, 3): 1, (0, 4): 2,  # spins (A, B, Cin, S, Cout)
        (1, 2): -1, (1, 3): 1, (1, 4): 2,
        (2, 3): 1, (2, 4): 2,
        (3, 4): -2}
FA_H = (0, 0, 0, 0, 0)


@dataclass
class Multiplier:
    """A w x w array multiplier as an Ising instance plus its named spin indices."""
    w: int
    n_spins: int
    edge_i: np.ndarray
    edge_j: np.ndarray
    edge_J: np.ndarray
    h: np.ndarray
    A: list[int]          # factor A spins, LSB first
    B: list[int]          # factor B spins, LSB first
    C: list[int]          # product spins, LSB first (2w of them)
    zeros: list[int]      # carry-in spins held at logical 0
    gates: list[tuple[str, tuple[int, ...]]]

    def instance(self, product: int | None = None) -> Instance:
        """Clamp the carry-ins to 0 and, if given, the product bits to `product`."""
        clamp = np.zeros(self.n_spins, dtype=np.int8)
        clamp[self.zeros] = -1
        if product is not None:
            if product < 0 or product >= (1 << (2 * self.w)):
                raise ValueError("product out of range")
            for k, s in enumerate(self.C):
                clamp[s] = 1 if (product >> k) & 1 else -1
        return Instance(self.n_spins, self.edge_i.copy(), self.edge_j.copy(), self.edge_J.copy(),
                        self.h.copy(), clamp, 0,
                        {"kind": "multiplier", "w": self.w, "product": product})

    def decode(self, spins: np.ndarray) -> tuple[int, int]:
        """Read A and B (as integers) from a configuration of +-1 spins."""
        a = sum(1 << k for k, s in enumerate(self.A) if spins[s] > 0)
        b = sum(1 << k for k, s in enumerate(self.B) if spins[s] > 0)
        return a, b


def multiplier(w: int) -> Multiplier:
    """Build the invertible w x w array multiplier.

    The paper gives the gates (Supplementary S4) but not the wiring. The wiring here is a
    ripple array of full adders: partial products p[i][j] = a_j AND b_i; row 1 adds
    p[1][j] to p[0][j+1]; row i >= 2 adds p[i][j] to the previous row's sums shifted by one,
    with the previous row's final carry as the top input. The first carry-in of each row and
    the top input of row 1's last adder are spins held at logical 0. That gives
    N = w (A) + w (B) + w^2 (AND outputs) + 2 w (w-1) (adder S, Cout) + w (zeros) = 3w^2 + w,
    which reproduces the spin counts of the paper's scaling study (N = 3/4 n^2 + 1/2 n with
    n = 2w product bits; Supplementary S5 and Table S3).
    Spin order is {product C}{carry-ins}{other internal spins}{B}{A} (Supplementary S6).
    """
    if w < 2:
        raise ValueError("w must be >= 2")
    # symbolic names first, numbered at the end in the paper's order
    names: list[str] = []

    def new(name: str) -> str:
        names.append(name)
        return name

    A = [new(f"a{j}") for j in range(w)]
    B = [new(f"b{i}") for i in range(w)]
    p = [[new(f"p{i}_{j}") for j in range(w)] for i in range(w)]
    gates: list[tuple[str, tuple[str, ...]]] = []
    for i in range(w):
        for j in range(w):
            gates.append(("AND", (A[j], B[i], p[i][j])))
    zeros: list[str] = []
    S: list[list[str]] = [[] for _ in range(w)]
    Co: list[list[str]] = [[] for _ in range(w)]
    for i in range(1, w):
        for j in range(w):
            x = p[i][j]
            if i == 1:
                if j < w - 1:
                    y = p[0][j + 1]
                else:
                    y = new(f"z{i}_top")
                    zeros.append(y)
            else:
                y = S[i - 1][j + 1] if j < w - 1 else Co[i - 1][w - 1]
            if j == 0:
                cin = new(f"z{i}_cin")
                zeros.append(cin)
            else:
                cin = Co[i][j - 1]
            s = new(f"s{i}_{j}")
            c = new(f"c{i}_{j}")
            S[i].append(s)
            Co[i].append(c)
            gates.append(("FA", (x, y, cin, s, c)))
    C = [p[0][0]] + [S[i][0] for i in range(1, w - 1)] + \
        [S[w - 1][j] for j in range(w)] + [Co[w - 1][w - 1]]
    assert len(C) == 2 * w
    assert len(names) == 3 * w * w + w, (len(names), 3 * w * w + w)
    # order: {C}{carry-ins}{internal}{B}{A}
    first = C + zeros
    tail = B + A
    middle = [n for n in names if n not in set(first) and n not in set(tail)]
    order = first + middle + tail
    idx = {n: k for k, n in enumerate(order)}
    N = len(order)
    Jd: dict[tuple[int, int], int] = {}
    h = np.zeros(N, dtype=np.int32)
    gates_idx: list[tuple[str, tuple[int, ...]]] = []
    for kind, spins in gates:
        ids = tuple(idx[s] for s in spins)
        gates_idx.append((kind, ids))
        Jg, hg = (AND_J, AND_H) if kind == "AND" else (FA_J, FA_H)
        for (a, b), v in Jg.items():
            u, t = ids[a], ids[b]
            key = (min(u, t), max(u, t))
            Jd[key] = Jd.get(key, 0) + v
        for a, v in enumerate(hg):
            h[ids[a]] += v
    keys = sorted(k for k, v in Jd.items() if v != 0)
    ei = np.array([k[0] for k in keys], dtype=np.int32)
    ej = np.array([k[1] for k in keys], dtype=np.int32)
    eJ = np.array([Jd[k] for k in keys], dtype=np.int32)
    return Multiplier(w, N, ei, ej, eJ, h, [idx[a] for a in A], [idx[b] for b in B],
                      [idx[c] for c in C], [idx[z] for z in zeros], gates_idx)


def primes_upto(n: int) -> list[int]:
    sieve = np.ones(n + 1, dtype=bool)
    sieve[:2] = False
    for k in range(2, int(math.isqrt(n)) + 1):
        if sieve[k]:
            sieve[k * k::k] = False
    return [int(v) for v in np.nonzero(sieve)[0]]


def draw_prime_products(count: int, max_factor: int = 255, seed: int = MASTER_SEED
                        ) -> list[tuple[int, int, int]]:
    """`count` products C = p*q of two primes p, q <= max_factor (8-bit primes), seeded."""
    ps = primes_upto(max_factor)
    g = _rng(seed, 0xFAC7, max_factor)
    out = []
    for _ in range(count):
        p, q = int(g.choice(ps)), int(g.choice(ps))
        out.append((p * q, p, q))
    return out


# ----------------------------------------------------------------------------------------
# Proposal pools and random configurations
# ----------------------------------------------------------------------------------------

def random_configs(n_spins: int, count: int, seed: int = MASTER_SEED, index: int = 0
                   ) -> np.ndarray:
    """`count` uniformly random +-1 configurations, int8 [count][n_spins]."""
    b = _rng(seed, 0x9001, n_spins, index).integers(0, 2, size=(count, n_spins), dtype=np.int8)
    return (2 * b - 1).astype(np.int8)


def pack_bits(spins: np.ndarray) -> np.ndarray:
    """Pack +-1 spins [..., N] into uint32 words [..., ceil(N/32)], bit (i % 32) of word
    i // 32 set when spin i is +1."""
    s = np.asarray(spins)
    N = s.shape[-1]
    NW = (N + 31) // 32
    bits = np.zeros(s.shape[:-1] + (NW * 32,), dtype=np.uint64)
    bits[..., :N] = (s > 0)
    bits = bits.reshape(s.shape[:-1] + (NW, 32))
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (bits * weights).sum(axis=-1).astype(np.uint32)


def unpack_bits(words: np.ndarray, N: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint32)
    bits = (w[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1
    bits = bits.reshape(w.shape[:-1] + (w.shape[-1] * 32,))[..., :N]
    return (2 * bits.astype(np.int8) - 1).astype(np.int8)


# ---------------------------------------------------------------------------------- IsingFormer
# Seeded parameters of the IsingFormer decoder (Methods, "IsingFormer architecture and
# training"; Supplementary S6). No trained weights exist here, so the parameters are random;
# they are rounded to bfloat16, the format the GPU library keeps them in, and both the library
# and the oracle take exactly these values.

@dataclass
class FormerShape:
    n_spins: int            # sequence length N
    d_model: int = 256
    n_heads: int = 4
    n_layers: int = 5
    d_ff: int = 1024


def former_param_shapes(s: FormerShape) -> list[tuple[str, tuple[int, ...]]]:
    """The parameters in their packing order (the order of the C ABI's weight array). Matrices
    are row-major [in][out]: y = x W + b."""
    d, F = s.d_model, s.d_ff
    out = [("tok_emb", (3, d)), ("w_beta", (d,)), ("b_beta", (d,))]
    for l in range(s.n_layers):
        out += [(f"l{l}.ln1_g", (d,)), (f"l{l}.ln1_b", (d,)), (f"l{l}.w_qkv", (d, 3 * d)),
                (f"l{l}.b_qkv", (3 * d,)), (f"l{l}.w_o", (d, d)), (f"l{l}.b_o", (d,)),
                (f"l{l}.ln2_g", (d,)), (f"l{l}.ln2_b", (d,)), (f"l{l}.w_1", (d, F)),
                (f"l{l}.b_1", (F,)), (f"l{l}.w_2", (F, d)), (f"l{l}.b_2", (d,))]
    out += [("lnf_g", (d,)), ("lnf_b", (d,)), ("w_out", (d, 2)), ("b_out", (2,))]
    return out


def bf16_round(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Round to bfloat16 (nearest, ties to even): the 16-bit patterns and their values."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
    v = (r.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return r, v.reshape(x.shape)


def former_weights(s: FormerShape, seed: int = MASTER_SEED, index: int = 0):
    """Random IsingFormer parameters, bfloat16-rounded: (dict of float64 arrays, packed uint16
    array in former_param_shapes order). Matrices ~ N(0, 1/fan_in), the token and beta
    embeddings ~ N(0, 1), layer-norm gains 1 + N(0, 0.1^2), biases ~ N(0, 0.1^2)."""
    g = _rng(seed, 0xF0, s.n_spins, index)
    vals, packed = {}, []
    for name, shape in former_param_shapes(s):
        if name.endswith("_g"):
            x = 1.0 + 0.1 * g.standard_normal(shape)
        elif name in ("tok_emb", "w_beta"):
            x = g.standard_normal(shape)
        elif len(shape) == 2:
            x = g.standard_normal(shape) / math.sqrt(shape[0])
        else:
            x = 0.1 * g.standard_normal(shape)
        r, v = bf16_round(x)
        vals[name] = v
        packed.append(r.reshape(-1))
    return vals, np.concatenate(packed)
