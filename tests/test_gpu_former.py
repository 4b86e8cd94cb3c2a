"""IsingFormer inference on the GPU (libptformer.so) against the float64 oracle
(oracle/former.py), at the paper's spin-glass and factorization shape (d_model 256, 4
heads, 5 layers, FFN 1024; Methods and Supplementary S6) with seeded bfloat16 weights.

Tolerance. The GPU rounds every matrix-product input (layer-norm, attention and GELU
outputs) to bfloat16, a relative error of at most 2^-9 each, and accumulates in FP32; the
oracle keeps float64 throughout. Over 5 residual blocks these roundings leave logit errors of
order 1e-2; the bound used is 0.05 + 0.02 |logit|, and for log q, a sum of N
log-probabilities whose errors add with random signs, 0.02 sqrt(N) + 0.01 |log q|."""
import numpy as np
import pytest

import instances as I
import oracle as O
from oracle import former as F

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _model(N, index=0, shape=None, attn_mode=0):
    from paper_2509_23043_gb300.former import Former
    shp = shape or I.FormerShape(n_spins=N)
    W, packed = I.former_weights(shp, index=index)
    return shp, W, Former(shp, packed, attn_mode=attn_mode)


@pytest.mark.parametrize("attn_mode", [0, 1, 2])
@pytest.mark.parametrize("N,B", [(37, 6), (200, 4), (300, 3)])
def test_score_matches_oracle(N, B, attn_mode):
    # attn_mode 0: tensor-core attention, scores and softmax fused for N = 200 (37 is not a
    # multiple of 8 and 300 exceeds one key tile: those take mode 2's path); 1: the streaming
    # FP32 kernel; 2: cuBLASLt scores and the softmax kernel
    shp, W, m = _model(N, index=N, attn_mode=attn_mode)
    g = np.random.default_rng(N)
    X = np.where(g.random((B, N)) < 0.5, 1, -1).astype(np.int8)
    beta = g.uniform(0.1, 3.0, B)
    lq, lg = m.score(torch.from_numpy(X).cuda(), torch.from_numpy(beta.astype(np.float32)).cuda(), logits=True)
    lg_o, lq_o = F.score(W, shp, X, beta.astype(np.float32).astype(np.float64))
    lg, lq = lg.cpu().numpy().astype(np.float64), lq.cpu().numpy().astype(np.float64)
    err = np.abs(lg - lg_o)
    print("max logit error", err.max(), "max |logit|", np.abs(lg_o).max(), "log q errors", np.abs(lq - lq_o))
    assert np.all(err <= 0.05 + 0.02 * np.abs(lg_o)), err.max()
    assert np.all(np.abs(lq - lq_o) <= 0.02 * np.sqrt(N) + 0.01 * np.abs(lq_o)), (lq, lq_o)


@pytest.mark.parametrize("N,B", [(37, 3), (200, 5), (64, 2)])
def test_tcgen05_projections_match_library_products(N, B):
    # Every projection by this library's tcgen05 kernels (proj_mode 2: bias, GELU and the
    # residual add in their epilogues) against cuBLASLt products and the GELU kernel
    # (proj_mode 1): the same bfloat16 operands and FP32 accumulation, so the paths differ by
    # accumulation order and by the rounding of the FFN activations (one rounding to bfloat16
    # in the kernel, two in the library path). Rows M = B N = 111, 1000 and 128: a partial
    # tile, several tiles with a ragged tail, one tile.
    from paper_2509_23043_gb300.former import Former
    shp = I.FormerShape(n_spins=N)
    W, packed = I.former_weights(shp, index=N + 1)
    tc = Former(shp, packed, proj_mode=2)
    lib = Former(shp, packed, proj_mode=1)
    g = np.random.default_rng(N + 7)
    X = torch.from_numpy(np.where(g.random((B, N)) < 0.5, 1, -1).astype(np.int8)).cuda()
    beta = torch.from_numpy(g.uniform(0.1, 3.0, B).astype(np.float32)).cuda()
    for _ in range(2):                        # two calls in a row on the same buffers
        lq0, lg0 = tc.score(X, beta, logits=True)
        lq1, lg1 = lib.score(X, beta, logits=True)
        tc.check()
        lg0, lg1 = lg0.cpu().numpy(), lg1.cpu().numpy()
        assert np.isfinite(lg0).all()
        d = np.abs(lg0 - lg1)
        print("tcgen05 vs library: max logit difference", d.max())
        assert d.max() < 0.02, d.max()
        assert np.abs(lq0.cpu().numpy() - lq1.cpu().numpy()).max() < 0.02 * np.sqrt(N)
        assert d.max() > 0                    # the two paths are distinct code
    lg_o, _ = F.score(W, shp, X.cpu().numpy(), beta.cpu().numpy().astype(np.float64))
    assert np.all(np.abs(lg0 - lg_o) <= 0.05 + 0.02 * np.abs(lg_o))


@pytest.mark.parametrize("N,B", [(8, 5), (64, 3), (136, 2), (200, 4), (256, 2), (200, 160)])
def test_fused_attention_matches_library_attention(N, B):
    # attn_mode 0: scores, causal softmax and P V in one tcgen05 kernel (one tile per 128
    # queries, the whole score row in TMEM, P through shared memory) against attn_mode 2
    # (cuBLASLt scores in FP32, the softmax kernel, cuBLASLt P V): the same bfloat16 queries,
    # keys and values and FP32 scores, the probabilities rounded to bfloat16 on both sides (the
    # fused kernel before normalising); N = 8 .. 256 covers one query tile, a ragged second
    # tile (136 = 128 + 8) and the largest key tile, and B = 160 at N = 200 gives every block
    # about eight tiles (both stages, both accumulators and the P buffer in turn); the logits
    # also agree with the float64 oracle
    from paper_2509_23043_gb300.former import Former
    shp = I.FormerShape(n_spins=N)
    W, packed = I.former_weights(shp, index=2 * N + 1)
    fused = Former(shp, packed, attn_mode=0)
    lib = Former(shp, packed, attn_mode=2)
    g = np.random.default_rng(N + 3)
    Xh = np.where(g.random((B, N)) < 0.5, 1, -1).astype(np.int8)
    bh = g.uniform(0.1, 3.0, B).astype(np.float32)
    X, beta = torch.from_numpy(Xh).cuda(), torch.from_numpy(bh).cuda()
    for _ in range(2):
        lq0, lg0 = fused.score(X, beta, logits=True)
        lq1, lg1 = lib.score(X, beta, logits=True)
        fused.check()
        lg0, lg1 = lg0.cpu().numpy(), lg1.cpu().numpy()
        assert np.isfinite(lg0).all()
        d = np.abs(lg0 - lg1)
        print("fused attention vs library attention: max logit difference", d.max())
        # each side rounds the probabilities to bfloat16 (2^-9 relative) at its own point and
        # sums in its own order: differences of order 1e-3, tails near 1e-2 over 64 000
        # logits; the bound of the projections comparison above
        assert d.max() < 0.02, d.max()
    lg_o, _ = F.score(W, shp, Xh, bh.astype(np.float64))
    print("fused attention vs the float64 oracle: max logit error", np.abs(lg0 - lg_o).max())
    assert np.all(np.abs(lg0 - lg_o) <= 0.05 + 0.02 * np.abs(lg_o))


def test_tcgen05_first_ffn_map_at_scale():
    # proj_mode 0 at 25600 rows (B = 128 configurations of N = 200): the first FFN map runs on
    # the tcgen05 kernel (200 tiles on the persistent grid), everything else on cuBLASLt; the
    # logits agree with the library path and with the float64 oracle on sampled rows
    from paper_2509_23043_gb300.former import Former
    N, B = 200, 128
    shp = I.FormerShape(n_spins=N)
    W, packed = I.former_weights(shp, index=3)
    auto = Former(shp, packed, proj_mode=0)
    lib = Former(shp, packed, proj_mode=1)
    g = np.random.default_rng(5)
    Xh = np.where(g.random((B, N)) < 0.5, 1, -1).astype(np.int8)
    bh = g.uniform(0.1, 3.0, B).astype(np.float32)
    X, beta = torch.from_numpy(Xh).cuda(), torch.from_numpy(bh).cuda()
    _, lg0 = auto.score(X, beta, logits=True)
    _, lg1 = lib.score(X, beta, logits=True)
    auto.check()
    lg0, lg1 = lg0.cpu().numpy(), lg1.cpu().numpy()
    d = np.abs(lg0 - lg1)
    print("tcgen05 first FFN map at 25600 rows: max logit difference", d.max())
    assert 0 < d.max() < 0.02
    rows = [0, 57, 127]
    lg_o, _ = F.score(W, shp, Xh[rows], bh[rows].astype(np.float64))
    assert np.all(np.abs(lg0[rows] - lg_o) <= 0.05 + 0.02 * np.abs(lg_o))


def _philox_u(seed, t, b, stream):
    w = O.philox([t, b, 6 << 24, stream], [seed & 0xFFFFFFFF, seed >> 32])[0]
    return (int(w) >> 8) * 2.0 ** -24


def test_sampling_matches_the_oracle_decisions():
    # every drawn spin is the threshold decision of the oracle's q(+1 | prefix) at the GPU's
    # own prefix, except within 0.02 of a tie; the first spins are the given prefix; the log q
    # the sampler reports (key/value-cache path) agrees with the scoring pass
    N, B, npre, seed, sid = 40, 24, 5, 0x1234_5678_9ABC, 7
    shp, W, m = _model(N, index=3, attn_mode=1)   # the scoring pass with FP32 attention, as the sampler's
    g = np.random.default_rng(11)
    beta = g.uniform(0.2, 2.5, B).astype(np.float32)
    pre = np.where(g.random((B, npre)) < 0.5, 1, -1).astype(np.int8)
    bt, pt_ = torch.from_numpy(beta).cuda(), torch.from_numpy(pre).cuda()
    out = torch.empty((B, N), dtype=torch.int8, device="cuda")
    lq = torch.empty(B, dtype=torch.float32, device="cuda")
    m.sample(bt, seed, sid, prefix=pt_, out=out, logq=lq)
    S = out.cpu().numpy()
    assert np.array_equal(S[:, :npre], pre)
    assert set(np.unique(S)) <= {-1, 1}
    lg_o, lq_o = F.score(W, shp, S, beta.astype(np.float64))
    p_plus = np.exp(F.log_softmax2(lg_o)[..., 1])
    near = 0
    for b in range(B):
        for t in range(npre, N):
            u = _philox_u(seed, t, b, sid)
            if abs(u - p_plus[b, t]) < 0.02:
                near += 1
                continue
            assert S[b, t] == (1 if u < p_plus[b, t] else -1), (b, t, u, p_plus[b, t])
    assert near < 0.05 * B * (N - npre)
    lq_gpu = lq.cpu().numpy().astype(np.float64)
    lq_s = m.score(torch.from_numpy(S).cuda(), bt).cpu().numpy().astype(np.float64)
    assert np.allclose(lq_gpu, lq_s, atol=1e-3 * np.sqrt(N), rtol=1e-4), (lq_gpu, lq_s)
    assert np.all(np.abs(lq_gpu - lq_o) <= 0.02 * np.sqrt(N) + 0.01 * np.abs(lq_o))
    # later calls with the same arrays replay the captured graph: the same seed gives the same
    # draw, another seed another one
    m.sample(bt, seed, sid, prefix=pt_, out=out, logq=lq)
    assert np.array_equal(out.cpu().numpy(), S)
    assert np.allclose(lq.cpu().numpy(), lq_gpu, atol=0, rtol=0)
    m.sample(bt, seed + 1, sid, prefix=pt_, out=out, logq=lq)
    assert not np.array_equal(out.cpu().numpy(), S)


@pytest.mark.parametrize("N,B", [(40, 24), (200, 16)])
def test_bfloat16_cache_sampling_matches_scoring(N, B):
    # attn_mode 0: the sampler's bfloat16 key/value cache takes the fused scoring kernel's
    # arithmetic (bfloat16 query, keys and values, FP32 scores, the same exponential, the
    # unnormalised probabilities rounded to bfloat16 before P V), so the log q it reports is
    # the scoring pass's up to summation order; every drawn spin is the oracle's threshold
    # decision at the GPU's own prefix except within 0.02 of a tie
    npre, seed, sid = 5, 0x2468_ACE0_1357, 3
    shp, W, m = _model(N, index=N + 9, attn_mode=0)
    g = np.random.default_rng(N + 21)
    beta = g.uniform(0.2, 2.5, B).astype(np.float32)
    pre = np.where(g.random((B, npre)) < 0.5, 1, -1).astype(np.int8)
    bt, pt_ = torch.from_numpy(beta).cuda(), torch.from_numpy(pre).cuda()
    out = torch.empty((B, N), dtype=torch.int8, device="cuda")
    lq = torch.empty(B, dtype=torch.float32, device="cuda")
    m.sample(bt, seed, sid, prefix=pt_, out=out, logq=lq)
    m.check()
    S = out.cpu().numpy()
    assert np.array_equal(S[:, :npre], pre)
    lq_gpu = lq.cpu().numpy().astype(np.float64)
    lq_s = m.score(torch.from_numpy(S).cuda(), bt).cpu().numpy().astype(np.float64)
    print("bfloat16-cache sampler vs scoring: max log q difference", np.abs(lq_gpu - lq_s).max())
    assert np.allclose(lq_gpu, lq_s, atol=1e-3 * np.sqrt(N), rtol=1e-4), (lq_gpu, lq_s)
    lg_o, lq_o = F.score(W, shp, S, beta.astype(np.float64))
    assert np.all(np.abs(lq_gpu - lq_o) <= 0.02 * np.sqrt(N) + 0.01 * np.abs(lq_o))
    p_plus = np.exp(F.log_softmax2(lg_o)[..., 1])
    near = 0
    for b in range(B):
        for t in range(npre, N):
            u = _philox_u(seed, t, b, sid)
            if abs(u - p_plus[b, t]) < 0.02:
                near += 1
                continue
            assert S[b, t] == (1 if u < p_plus[b, t] else -1), (b, t, u, p_plus[b, t])
    assert near < 0.05 * B * (N - npre)


def test_sampled_frequencies_follow_q():
    # a small model (d 64, one head, 2 layers) over N = 6 spins: the frequencies of 40000
    # GPU draws follow the exact q(x | beta) of the oracle over all 64 configurations, within
    # 5 sigma of the multinomial noise (plus the bfloat16 model error, below 1e-2 in total
    # variation on these weights)
    shp = I.FormerShape(n_spins=6, d_model=64, n_heads=1, n_layers=2, d_ff=128)
    shp, W, m = _model(6, index=5, shape=shp)
    X = np.array([[1 if (k >> (5 - i)) & 1 else -1 for i in range(6)] for k in range(64)], np.int8)
    _, lq = F.score(W, shp, X, np.full(64, 1.4))
    q = np.exp(lq)
    n = 40000
    S, _ = m.sample(torch.full((n,), 1.4, dtype=torch.float32, device="cuda"), 99, 0)
    S = S.cpu().numpy()
    code = ((S > 0).astype(np.int64) << np.arange(6)[::-1]).sum(1)
    emp = np.bincount(code, minlength=64) / n
    tv = 0.5 * np.abs(emp - q).sum()
    assert tv < 5 * 0.5 * np.sum(np.sqrt(q * (1 - q) / n)) + 0.01, tv


@pytest.mark.parametrize("shape", [
    I.FormerShape(n_spins=1),                                            # one spin: one key
    I.FormerShape(n_spins=9, d_model=64, n_heads=1, n_layers=0, d_ff=128),  # no blocks at all
    I.FormerShape(n_spins=16, d_model=64, n_heads=1, n_layers=1, d_ff=64),  # one block of width 64
])
def test_degenerate_shapes_score_and_sample(shape):
    # B = 1: a single spin (the start token alone, attention over one key), a model without
    # blocks (embedding, final layer norm and head) and one block of width 64 (one head, the
    # fused attention with H = 1); scoring against the float64 oracle, and the sampler's log q
    # against the scoring pass
    N = shape.n_spins
    shp, W, m = _model(N, index=77, shape=shape)
    X = np.ones((1, N), np.int8)
    X[0, ::2] = -1
    beta = np.array([1.3], np.float32)
    bt = torch.from_numpy(beta).cuda()
    lq, lg = m.score(torch.from_numpy(X).cuda(), bt, logits=True)
    lg_o, lq_o = F.score(W, shp, X, beta.astype(np.float64))
    assert np.all(np.abs(lg.cpu().numpy() - lg_o) <= 0.05 + 0.02 * np.abs(lg_o))
    assert abs(float(lq.cpu()[0]) - lq_o[0]) <= 0.02 * np.sqrt(N) + 0.01 * abs(lq_o[0])
    S, lqs = m.sample(bt, 5, 1)
    m.check()
    S = S.cpu().numpy()
    assert S.shape == (1, N) and set(np.unique(S)) <= {-1, 1}
    lq_s = m.score(torch.from_numpy(S).cuda(), bt).cpu().numpy()
    assert abs(float(lqs.cpu()[0]) - lq_s[0]) <= 1e-3 * np.sqrt(N) + 1e-4 * abs(lq_s[0])


def test_invalid_calls_are_rejected():
    # a width that is not 64 per head, an empty batch, a prefix longer than N and a sequence
    # whose per-head scores exceed the sampler's shared memory are refused with a status; the
    # model answers normally afterwards
    from paper_2509_23043_gb300 import PT_EINVAL, PT_ENOTSUP, PTError
    from paper_2509_23043_gb300.former import Former
    bad = I.FormerShape(n_spins=8, d_model=96, n_heads=1, n_layers=1, d_ff=64)
    _, packed = I.former_weights(bad)
    with pytest.raises(PTError) as e:
        Former(bad, packed)
    assert e.value.status == PT_EINVAL
    shp, W, m = _model(8, index=1, shape=I.FormerShape(n_spins=8, d_model=64, n_heads=1, n_layers=1, d_ff=64))
    beta = torch.ones(2, dtype=torch.float32, device="cuda")
    with pytest.raises(PTError) as e:
        m.score(torch.empty((0, 8), dtype=torch.int8, device="cuda"), beta[:0])
    assert e.value.status == PT_EINVAL
    with pytest.raises(PTError) as e:
        m.sample(beta, 1, 0, prefix=torch.ones((2, 9), dtype=torch.int8, device="cuda"))
    assert e.value.status == PT_EINVAL
    big = I.FormerShape(n_spins=4096, d_model=256, n_heads=4, n_layers=1, d_ff=64)
    _, _, mb = _model(4096, index=2, shape=big)
    with pytest.raises(PTError) as e:
        mb.sample(torch.ones(1, dtype=torch.float32, device="cuda"), 1, 0)
    assert e.value.status == PT_ENOTSUP
    X = np.where(np.arange(16).reshape(2, 8) % 3 == 0, 1, -1).astype(np.int8)
    lq = m.score(torch.from_numpy(X).cuda(), beta).cpu().numpy()
    _, lq_o = F.score(W, shp, X, np.ones(2))
    assert np.all(np.abs(lq - lq_o) <= 0.02 * np.sqrt(8) + 0.01 * np.abs(lq_o))
