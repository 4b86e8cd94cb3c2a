"""The seeded input generators (the input recipe): EA lattices in canonical bond order with
J = -1 at p = 0.5, geometric ladders, 8-bit prime products, and the bit packing of pools."""
import numpy as np

import instances as I


def test_ea_bonds_are_canonical_and_periodic():
    L = 5
    inst = I.ea_instance(L, index=3)
    N = L ** 3
    assert inst.n_spins == N and inst.lattice_L == L and len(inst.edge_J) == 3 * N
    for n in range(N):
        x, y, z = n % L, (n // L) % L, n // (L * L)
        want = [((x + 1) % L) + L * (y + L * z), x + L * (((y + 1) % L) + L * z),
                x + L * (y + L * ((z + 1) % L))]
        assert list(inst.edge_i[3 * n:3 * n + 3]) == [n, n, n]
        assert list(inst.edge_j[3 * n:3 * n + 3]) == want
    assert set(np.unique(inst.edge_J)) <= {-1, 1}
    assert inst.h is None and inst.clamp is None


def test_ea_couplings_are_fair_and_seeded():
    big = I.ea_instance(16, index=0)
    frac = float(np.mean(big.edge_J < 0))
    assert abs(frac - 0.5) < 4 * np.sqrt(0.25 / big.edge_J.size)       # p = 0.5 within 4 sigma
    again = I.ea_instance(16, index=0)
    other = I.ea_instance(16, index=1)
    assert np.array_equal(big.edge_J, again.edge_J) and not np.array_equal(big.edge_J, other.edge_J)
    assert np.all(I.ea_instance(4, ferro=True).edge_J == 1)


def test_geometric_ladder_ends_and_ratio():
    b = I.geometric_betas(0.1, 3.0, 32)
    assert b[0] == 0.1 and abs(b[-1] - 3.0) < 1e-12 and np.all(np.diff(b) > 0)
    r = b[1:] / b[:-1]
    assert np.allclose(r, r[0])


def test_prime_products_use_primes_up_to_the_bound():
    ps = set(I.primes_upto(255))
    assert len(ps) == 54 and 2 in ps and 251 in ps and 255 not in ps and 1 not in ps
    for C, p, q in I.draw_prime_products(200):
        assert p in ps and q in ps and C == p * q
    assert I.draw_prime_products(5) == I.draw_prime_products(5)


def test_pack_and_unpack_are_inverse():
    rng = np.random.default_rng(7)
    for N in (1, 31, 32, 33, 100):
        s = (2 * rng.integers(0, 2, size=(6, N)) - 1).astype(np.int8)
        words = I.pack_bits(s)
        assert words.shape[-1] == (N + 31) // 32
        assert np.array_equal(I.unpack_bits(words, N), s)
