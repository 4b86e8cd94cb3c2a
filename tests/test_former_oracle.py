"""Pins of the IsingFormer oracle (oracle/former.py) against structural facts of a causal
autoregressive decoder (Methods, "IsingFormer architecture and training"; Supplementary S6),
on small shapes where they can be checked exhaustively. A misaligned start token, a leak of
the predicted spin into its own context, a broken causal mask, a positional code or a beta
embedding entered at the wrong place each fail one of them."""
import itertools
import math

import numpy as np
import pytest

import instances as I
from oracle import former as F

SMALL = I.FormerShape(n_spins=6, d_model=16, n_heads=2, n_layers=2, d_ff=32)


def _all_configs(N):
    return np.array(list(itertools.product([-1, 1], repeat=N)), dtype=np.int8)


@pytest.mark.parametrize("beta", [0.0, 0.7, 3.1])
def test_autoregressive_probabilities_sum_to_one(beta):
    # q(x | beta) = prod_t q(x_t | x_<t) sums to 1 over all 2^N configurations only if spin t
    # is predicted from spins 0 .. t-1 alone
    W, _ = I.former_weights(SMALL, index=1)
    X = _all_configs(SMALL.n_spins)
    _, lq = F.score(W, SMALL, X, np.full(len(X), beta))
    assert abs(np.exp(lq).sum() - 1.0) < 1e-12


def test_outputs_are_causal():
    # the logits at position t do not change when spins t .. N-1 change
    W, _ = I.former_weights(SMALL, index=2)
    g = np.random.default_rng(4)
    X = np.where(g.random((8, SMALL.n_spins)) < 0.5, 1, -1).astype(np.int8)
    beta = g.uniform(0, 3, 8)
    base, _ = F.score(W, SMALL, X, beta)
    for t in range(SMALL.n_spins):
        Y = X.copy()
        Y[:, t:] = -Y[:, t:]
        other, _ = F.score(W, SMALL, Y, beta)
        assert np.allclose(base[:, :t + 1], other[:, :t + 1], atol=1e-12, rtol=0)
        if t + 1 < SMALL.n_spins:
            assert not np.allclose(base[:, t + 1:], other[:, t + 1:])


def test_first_position_sees_only_the_start_token_and_beta():
    W, _ = I.former_weights(SMALL, index=3)
    X = _all_configs(SMALL.n_spins)
    logits, _ = F.score(W, SMALL, X, np.full(len(X), 1.3))
    assert np.allclose(logits[:, 0], logits[0, 0], atol=1e-13, rtol=0)


def test_beta_embedding_is_added_to_every_position():
    # e_beta = W_beta beta + b_beta is added to the token embedding at every position: moving a
    # constant vector from b_beta into the token embeddings changes no output
    W, _ = I.former_weights(SMALL, index=4)
    c = np.random.default_rng(5).standard_normal(SMALL.d_model)
    W2 = dict(W, tok_emb=W["tok_emb"] + c, b_beta=W["b_beta"] - c)
    X = _all_configs(SMALL.n_spins)[::5]
    beta = np.linspace(0.1, 2.0, len(X))
    assert np.allclose(F.score(W, SMALL, X, beta)[0], F.score(W2, SMALL, X, beta)[0], atol=1e-10)
    # and a model whose beta weights are zero ignores beta
    W3 = dict(W, w_beta=np.zeros(SMALL.d_model))
    a, _ = F.score(W3, SMALL, X, np.full(len(X), 0.2))
    b, _ = F.score(W3, SMALL, X, np.full(len(X), 2.7))
    assert np.allclose(a, b, atol=1e-13, rtol=0)


def test_positional_encoding_values():
    pe = F.positional_encoding(5, 8)
    assert np.allclose(pe[0], [0, 1, 0, 1, 0, 1, 0, 1], atol=0)
    assert math.isclose(pe[3, 0], math.sin(3.0)) and math.isclose(pe[3, 1], math.cos(3.0))
    assert math.isclose(pe[2, 6], math.sin(2.0 / 10000 ** 0.75))


def test_layerless_model_closed_form():
    # with no transformer layers the logit of spin t is LN(E[tok] + e_beta + PE[t]) W_out +
    # b_out; for d = 2 the layer norm maps any vector with distinct entries to +-1 (eps aside)
    shp = I.FormerShape(n_spins=3, d_model=2, n_heads=1, n_layers=0, d_ff=2)
    W = {"tok_emb": np.array([[0.5, -0.5], [2.0, 1.0], [0.0, 3.0]]), "w_beta": np.array([1.0, 0.0]),
         "b_beta": np.array([0.0, 0.25]), "lnf_g": np.ones(2), "lnf_b": np.zeros(2),
         "w_out": np.array([[1.0, -2.0], [0.5, 0.0]]), "b_out": np.array([0.1, 0.2])}
    x = np.array([[1, -1, 1]], dtype=np.int8)
    logits, _ = F.score(W, shp, x, np.array([0.5]))
    # position 0: start token [0, 3] + [0.5, 0.25] + PE[0] = [0, 1] -> [0.5, 4.25] -> LN -> [-1, 1]
    # position 1: token of +1 [2, 1] + [0.5, 0.25] + [sin 1, cos 1] -> first entry larger -> [1, -1]
    for t, z in ((0, np.array([-1.0, 1.0])), (1, np.array([1.0, -1.0]))):
        s = 1.0 / math.sqrt(1.0 + F.LN_EPS)
        assert np.allclose(logits[0, t], s * z @ W["w_out"] + W["b_out"], atol=1e-12)


def test_sampling_follows_q():
    # with uniform u the sampled configurations follow q(x | beta); total variation within
    # 5 sigma of the multinomial noise over 64 states
    W, _ = I.former_weights(SMALL, index=6)
    X = _all_configs(SMALL.n_spins)
    beta = 0.9
    _, lq = F.score(W, SMALL, X, np.full(len(X), beta))
    q = np.exp(lq)
    n = 20000
    u = np.random.default_rng(7).random((n, SMALL.n_spins))
    S, lq_s, _ = F.sample(W, SMALL, np.full(n, beta), u)
    code = ((S > 0).astype(np.int64) << np.arange(SMALL.n_spins)[::-1]).sum(1)
    emp = np.bincount(code, minlength=64) / n
    tv = 0.5 * np.abs(emp - q).sum()
    assert tv < 5 * 0.5 * np.sum(np.sqrt(q * (1 - q) / n)), tv
    # the log q that sampling reports is the score of what it drew
    _, lq_chk = F.score(W, SMALL, S[:50], np.full(50, beta))
    assert np.allclose(lq_s[:50], lq_chk, atol=1e-12)


def test_sampling_keeps_the_prefix():
    # the first spins (the product and carry bits of the factorization order) are given
    W, _ = I.former_weights(SMALL, index=8)
    g = np.random.default_rng(9)
    pre = np.where(g.random((10, 2)) < 0.5, 1, -1).astype(np.int8)
    S, lq, _ = F.sample(W, SMALL, np.full(10, 1.1), g.random((10, SMALL.n_spins)), prefix=pre)
    assert np.array_equal(S[:, :2], pre)
    _, lq_chk = F.score(W, SMALL, S, np.full(10, 1.1))
    assert np.allclose(lq, lq_chk, atol=1e-12)


@pytest.mark.parametrize("shp", [SMALL, I.FormerShape(n_spins=9, d_model=64, n_heads=4, n_layers=3, d_ff=256)])
def test_blocks_match_the_library_transformer_layer(shp):
    # the pre-layer-norm decoder blocks (causal multi-head attention, GELU FFN, residuals,
    # final layer norm and linear head) are PyTorch's nn.TransformerEncoderLayer with
    # norm_first, exact GELU, no dropout and a causal mask: the oracle's logits equal the
    # library stack's on the same embedded input, in float64. A transposed operand, a head
    # split or scale, a residual or a layer norm in the wrong place each break the equality.
    torch = pytest.importorskip("torch")
    nn = torch.nn
    W, _ = I.former_weights(shp, index=5)
    d, H, F_ = shp.d_model, shp.n_heads, shp.d_ff
    g = np.random.default_rng(9)
    B, N = 3, shp.n_spins
    X = np.where(g.random((B, N)) < 0.5, 1, -1).astype(np.int8)
    beta = g.uniform(0.0, 4.0, B)
    logits, _ = F.score(W, shp, X, beta)

    tok = F.input_tokens(X)
    h = (W["tok_emb"][tok] + (beta[:, None] * W["w_beta"] + W["b_beta"])[:, None, :]
         + F.positional_encoding(N, d)[None])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).double()
    layers = []
    for l in range(shp.n_layers):
        p = f"l{l}."
        lay = nn.TransformerEncoderLayer(d, H, dim_feedforward=F_, dropout=0.0, activation="gelu",
                                         layer_norm_eps=F.LN_EPS, batch_first=True, norm_first=True)
        lay = lay.double().eval()
        with torch.no_grad():
            lay.self_attn.in_proj_weight.copy_(t(W[p + "w_qkv"].T))
            lay.self_attn.in_proj_bias.copy_(t(W[p + "b_qkv"]))
            lay.self_attn.out_proj.weight.copy_(t(W[p + "w_o"].T))
            lay.self_attn.out_proj.bias.copy_(t(W[p + "b_o"]))
            lay.linear1.weight.copy_(t(W[p + "w_1"].T))
            lay.linear1.bias.copy_(t(W[p + "b_1"]))
            lay.linear2.weight.copy_(t(W[p + "w_2"].T))
            lay.linear2.bias.copy_(t(W[p + "b_2"]))
            lay.norm1.weight.copy_(t(W[p + "ln1_g"]))
            lay.norm1.bias.copy_(t(W[p + "ln1_b"]))
            lay.norm2.weight.copy_(t(W[p + "ln2_g"]))
            lay.norm2.bias.copy_(t(W[p + "ln2_b"]))
        layers.append(lay)
    mask = torch.triu(torch.ones(N, N, dtype=torch.bool), diagonal=1)
    with torch.no_grad():
        z = t(h)
        for lay in layers:
            z = lay(z, src_mask=mask)
        z = torch.nn.functional.layer_norm(z, (d,), t(W["lnf_g"]), t(W["lnf_b"]), eps=F.LN_EPS)
        ref = (z @ t(W["w_out"]) + t(W["b_out"])).numpy()
    assert np.abs(logits - ref).max() < 1e-10
