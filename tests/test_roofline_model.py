"""The roofline's algorithmic count uses the expected number of plane blocks a bit-sliced word
needs (bench.blocks_for). Pinned here by simulating the lazy MSB-first comparison of uniform
32-bit draws with random thresholds, walker by walker. The IsingFormer's byte counts (the
sampler's key/value cache, the scoring pass's activations) are pinned against step-by-step and
kernel-by-kernel enumerations."""
import numpy as np
import pytest

import bench


def _simulated_blocks(n_und, words, rng):
    # a walker is decided at the first plane (MSB first) where u and T differ
    u = rng.integers(0, 2 ** 32, size=(words, n_und), dtype=np.uint64)
    t = rng.integers(0, 2 ** 32, size=(words, n_und), dtype=np.uint64)
    diff = u ^ t
    # planes needed = 32 - bit_length(diff) + 1 (first differing bit from the top); ties: 32
    bl = np.zeros_like(diff)
    x = diff.copy()
    while np.any(x):
        nz = x > 0
        bl[nz] += 1
        x >>= np.uint64(1)
    planes = np.where(diff > 0, 33 - bl, 32)
    need = planes.max(axis=1)                       # the word waits for its last walker
    return np.ceil(need / 4.0).mean()


@pytest.mark.parametrize("n_und", [1, 3, 10, 32])
def test_expected_blocks_match_a_simulation_of_the_lazy_compare(n_und):
    rng = np.random.default_rng(0xB10C + n_und)
    sim = _simulated_blocks(n_und, 20000, rng)
    exact = float(bench.blocks_for([n_und])[0])
    assert sim == pytest.approx(exact, abs=0.02), (sim, exact)


def test_expected_blocks_closed_values():
    # one walker: sum_k 2^-4k over k = 0..7; no walker: no block
    assert bench.blocks_for([1])[0] == pytest.approx(sum(16.0 ** -k for k in range(8)))
    assert bench.blocks_for([0])[0] == 0.0
    assert 1.9 < bench.blocks_for([32])[0] < 2.1      # the Gibbs case: every walker compares


def test_sampling_cache_bytes_match_a_step_by_step_count():
    # the sampler's roofline counts L B 2d e (N(N+1)/2 + N) cache bytes per call; counted here
    # step by step: at step t every layer appends row t and reads rows 0..t of each
    # configuration, 2d values of e bytes per row
    import instances as I
    for N, B, e in ((200, 1024, 2), (37, 8, 4)):
        shp = I.FormerShape(n_spins=N)
        row = 2 * shp.d_model * e
        total = sum(shp.n_layers * B * row * ((t + 1) + 1) for t in range(N))
        got = bench.sample_roofline(shp, B, 1.0, elem_bytes=e)["bytes_per_call"]
        assert got == total


def test_scoring_activation_bytes_match_a_kernel_by_kernel_count():
    # the scoring pass's HBM view counts the bytes its kernels pass to one another; listed here
    # kernel by kernel (buffer elements read and written, bytes per element): FP32 residual
    # stream h [M][d], bfloat16 norm output a [M][d], QKV [M][3d], attention output o [M][d],
    # FFN activations g [M][F]
    import instances as I
    shp = I.FormerShape(n_spins=200)
    B = 1024
    M, d, F, L = B * shp.n_spins, shp.d_model, shp.d_ff, shp.n_layers
    h, a, qkv, o, g = 4 * M * d, 2 * M * d, 2 * M * 3 * d, 2 * M * d, 2 * M * F
    total = h                                           # embedding writes h
    total += a                                          # ... and the first block's norm output
    for layer in range(L):
        if layer > 0:
            total += h + a                              # first layer norm
        total += a + qkv                                # QKV product
        total += qkv + o                                # fused attention
        total += o + 2 * h                              # output map into the residual stream
        total += h + a                                  # second layer norm
        total += a + g                                  # first FFN map with GELU
        total += g + 2 * h                              # second FFN map into the stream
    total += h                                          # head reads h
    got = bench.score_hbm_view(shp, B, 1.0)["bytes_per_call"]
    assert got == total
