"""The roofline's algorithmic count uses the expected number of plane blocks a bit-sliced word
needs (bench.blocks_for). Pinned here by simulating the lazy MSB-first comparison of uniform
32-bit draws with random thresholds, walker by walker."""
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
