"""IsingFormer inference restated in plain numpy float64 (Methods, "IsingFormer architecture
and training"; Supplementary S6, "Trained IsingFormers and proposal generation").

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the benchmark's CPU-baseline leg. The
GPU library never imports it.

The model is a decoder-only transformer over spin tokens: it gives q(x | beta), the
probability of a configuration x at inverse temperature beta, as the product of next-token
probabilities. What the paper fixes:
  - a two-token spin vocabulary; d_model = 256, 4 heads, 5 layers, FFN 4 d_model (the 3D
    spin-glass and factorization model), causal masked self-attention;
  - sinusoidal positional encodings (Vaswani et al.);
  - the beta embedding e_beta = W_beta beta + b_beta, added to the token embedding at every
    position, before the positional encoding;
  - factorization order {C}{carry}{multiplier}{B}{A}, C and the carry-ins given as the first
    tokens when sampling (a clamped prefix).
Readings where it is silent (each marked R below):
  R1 spin -1 is token 0 and +1 is token 1; a start token (2) fills input position 0, so the
     output at position t predicts spin t from spins 0 .. t-1;
  R2 pre-layer-norm blocks (h += Attn(LN(h)); h += FFN(LN(h))), layer norm with eps 1e-5,
     a final layer norm, then a linear head to two logits;
  R3 GELU in its erf form between the two FFN maps;
  R4 sampling draws spin t = +1 iff u_t < P(+1 | prefix), u_t uniform in [0, 1).
There are no trained weights, so no output of the paper's models can be compared. The pins
(tests/test_former_oracle.py) are the model's structural facts (normalisation, causality,
the start token, the positional code, a layer-free closed form) and, for the decoder blocks,
a library routine: PyTorch's nn.TransformerEncoderLayer with pre-layer-norm, exact GELU and
a causal mask gives the same logits in float64.
"""
from __future__ import annotations

import math

import numpy as np

LN_EPS = 1e-5


def positional_encoding(N: int, d: int) -> np.ndarray:
    """PE[t, 2i] = sin(t / 10000^(2i/d)), PE[t, 2i+1] = cos(t / 10000^(2i/d))."""
    t = np.arange(N, dtype=np.float64)[:, None]
    i = np.arange(d // 2, dtype=np.float64)[None, :]
    ang = t / np.power(10000.0, 2.0 * i / d)
    pe = np.zeros((N, d))
    pe[:, 0::2] = np.sin(ang)
    pe[:, 1::2] = np.cos(ang)
    return pe


def layer_norm(x, g, b):
    mu = x.mean(-1, keepdims=True)
    var = ((x - mu) ** 2).mean(-1, keepdims=True)
    return (x - mu) / np.sqrt(var + LN_EPS) * g + b


def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def input_tokens(spins: np.ndarray) -> np.ndarray:
    """R1: [start, tok(x_0), ..., tok(x_{N-2})] for each row of spins [B][N]."""
    B, N = spins.shape
    tok = np.empty((B, N), dtype=np.int64)
    tok[:, 0] = 2
    tok[:, 1:] = (spins[:, :-1] > 0).astype(np.int64)
    return tok


def forward(W: dict, shape, tok: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Logits [B][T][2] for input tokens [B][T] (T <= N) at inverse temperatures beta [B]."""
    d, H, L = shape.d_model, shape.n_heads, shape.n_layers
    dh = d // H
    B, T = tok.shape
    e_beta = beta[:, None] * W["w_beta"][None, :] + W["b_beta"][None, :]          # [B][d]
    h = W["tok_emb"][tok] + e_beta[:, None, :] + positional_encoding(T, d)[None]   # [B][T][d]
    future = np.triu(np.ones((T, T), dtype=bool), k=1)                             # key s > t
    for l in range(L):
        p = f"l{l}."
        a = layer_norm(h, W[p + "ln1_g"], W[p + "ln1_b"])
        qkv = a @ W[p + "w_qkv"] + W[p + "b_qkv"]
        q, k, v = qkv[..., :d], qkv[..., d:2 * d], qkv[..., 2 * d:]
        o = np.zeros_like(q)
        for j in range(H):
            sl = slice(j * dh, (j + 1) * dh)
            s = q[..., sl] @ np.swapaxes(k[..., sl], 1, 2) / math.sqrt(dh)        # [B][T][T]
            s = np.where(future[None], -np.inf, s)
            s = s - s.max(-1, keepdims=True)
            w = np.exp(s)
            w /= w.sum(-1, keepdims=True)
            o[..., sl] = w @ v[..., sl]
        h = h + o @ W[p + "w_o"] + W[p + "b_o"]
        f = layer_norm(h, W[p + "ln2_g"], W[p + "ln2_b"])
        h = h + gelu(f @ W[p + "w_1"] + W[p + "b_1"]) @ W[p + "w_2"] + W[p + "b_2"]
    z = layer_norm(h, W["lnf_g"], W["lnf_b"])
    return z @ W["w_out"] + W["b_out"]


def log_softmax2(logits):
    m = logits.max(-1, keepdims=True)
    return logits - m - np.log(np.exp(logits - m).sum(-1, keepdims=True))


def score(W: dict, shape, spins: np.ndarray, beta: np.ndarray):
    """Teacher-forced logits [B][N][2] and log q(x | beta) [B] of configurations spins [B][N]."""
    logits = forward(W, shape, input_tokens(spins), beta)
    lp = log_softmax2(logits)
    idx = (spins > 0).astype(np.int64)
    return logits, np.take_along_axis(lp, idx[..., None], -1)[..., 0].sum(-1)


def sample(W: dict, shape, beta: np.ndarray, u: np.ndarray, prefix: np.ndarray | None = None):
    """Autoregressive sampling (R4): spin t = +1 iff u[b, t] < P(+1 | spins < t); the first
    prefix.shape[1] spins are given (the clamped prefix). Returns spins [B][N], log q [B] and
    P(+1) [B][N] at each step. Recomputes the prefix at every step: slow, plain."""
    B, N = u.shape
    spins = np.zeros((B, N), dtype=np.int8)
    npre = 0 if prefix is None else prefix.shape[1]
    p_plus = np.zeros((B, N))
    logq = np.zeros(B)
    for t in range(N):
        tok = np.empty((B, t + 1), dtype=np.int64)
        tok[:, 0] = 2
        tok[:, 1:] = (spins[:, :t] > 0)
        lp = log_softmax2(forward(W, shape, tok, beta)[:, t, :])
        p_plus[:, t] = np.exp(lp[:, 1])
        if t < npre:
            s = prefix[:, t].astype(np.int8)
        else:
            s = np.where(u[:, t] < p_plus[:, t], 1, -1).astype(np.int8)
        spins[:, t] = s
        logq += np.where(s > 0, lp[:, 1], lp[:, 0])
    return spins, logq, p_plus
