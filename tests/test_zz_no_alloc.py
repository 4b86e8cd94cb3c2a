"""The allocation-free state read (pt_read_state_noalloc).

Some callers cannot allocate device memory while they run: a latency-bounded host loop
that keeps cudaMalloc/cudaFree (and the synchronisation they can cause) out of its steady
state, or a process that budgets all device memory up front. pt_read_state_noalloc gives
them the same result as pt_read_state through a fixed library-owned device buffer. These
tests call it through the C ABI and compare it with pt_read_state on two calls in a row.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import instances as I
import paper_2509_23043_gb300 as pt

pytestmark = pytest.mark.gpu


def _compare_twice(ctx, steps):
    for _ in range(2):
        pt.run_cycles(ctx, steps)
        for k in range(ctx.n):
            s_ref, E_ref = pt.read_state(ctx, k)
            s_new, E_new = pt.read_state_noalloc(ctx, k)
            assert np.array_equal(s_new, s_ref)       # integer results: bit-exact
            assert np.array_equal(E_new, E_ref)


def test_noalloc_read_matches_lattice_batch():
    insts = [I.ea_instance(L, index=900 + L) for L in (6, 7, 10)]
    betas = [I.geometric_betas(0.1, 3.0, R) for R in (16, 24, 40)]
    ctx = pt.create_instances(insts, betas, pt.Config(seed=21), instance_ids=[5, 6, 7])
    _compare_twice(ctx, 9)


def test_noalloc_read_matches_graph_engine():
    mult = I.multiplier(5)
    inst = mult.instance(23 * 29)
    ctx = pt.create_instances([inst], [I.geometric_betas(0.05, 5.0, 18)],
                              pt.Config(update=pt.GIBBS, seed=3), instance_ids=[667])
    _compare_twice(ctx, 11)


def test_noalloc_rejects_sizes_beyond_its_buffer():
    inst = I.ea_instance(18, index=1)                 # N = 5832, R = 48: 279936 bytes
    ctx = pt.create_instances([inst], [I.geometric_betas(0.2, 2.0, 48)], pt.Config(seed=1))
    with pytest.raises(pt.PTError) as e:
        pt.read_state_noalloc(ctx, 0)
    assert e.value.status == pt.PT_ENOTSUP
    assert "exceeds" in str(e.value)
    s, E = pt.read_state(ctx, 0)                      # the allocating path still serves it
    assert s.shape == (48, 5832)


def _cudart():
    import ctypes
    # the runtime libpt.so is linked against; dlopen by soname returns the loaded copy
    for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("CUDA runtime library not found")


def _pool_high_water(rt, pool, reset=False):
    import ctypes
    kUsedMemHigh = 0x8                                  # cudaMemPoolAttrUsedMemHigh
    v = ctypes.c_uint64(0)
    if reset:
        assert rt.cudaMemPoolSetAttribute(pool, kUsedMemHigh, ctypes.byref(v)) == 0
        return 0
    assert rt.cudaMemPoolGetAttribute(pool, kUsedMemHigh, ctypes.byref(v)) == 0
    return v.value


def test_noalloc_read_allocates_nothing():
    # The point of the entry point: no device allocation. pt_read_state takes its temporary
    # buffer from the device's default memory pool (cudaMallocAsync), so the pool's
    # high-water mark above the context's own memory rises during that call; during
    # pt_read_state_noalloc it must not rise at all.
    import ctypes
    rt = _cudart()
    inst = I.ea_instance(8, index=3)
    ctx = pt.create_instances([inst], [I.geometric_betas(0.1, 3.0, 32)], pt.Config(seed=4),
                              instance_ids=[11])
    pt.run_cycles(ctx, 5)
    pt.read_state_noalloc(ctx, 0)                       # the first call does its look-up
    dev = ctypes.c_int(0)
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p(0)
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev.value) == 0
    cur = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, 0x7, ctypes.byref(cur)) == 0   # UsedMemCurrent
    base = cur.value                                    # the context's own memory
    _pool_high_water(rt, pool, reset=True)              # high-water := current use
    for _ in range(3):
        pt.read_state_noalloc(ctx, 0)
    assert _pool_high_water(rt, pool) == base
    pt.read_state(ctx, 0)
    assert _pool_high_water(rt, pool) > base            # the allocating path does allocate
