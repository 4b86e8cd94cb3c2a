"""The multi-rank path on CPU: world_size 2 over gloo, one process per rank.

Instances shard across ranks with no collective in the data path; each rank runs its shard
(here through the oracle, since this machine has no GPU) and the job's time is the max over
ranks. These tests check that a sharded run reproduces the unsharded one instance by
instance (random streams are keyed by the global instance id, not by rank or slot), that
the ragged split is identical on every rank, disjoint and complete, and that the timing
reduction takes the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import instances as I
from paper_2509_23043_gb300 import shard

WORLD = 2
PER_RANK = 3
L, R, CYCLES, P = 4, 8, 25, 4


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_instance(gid: int):
    import oracle as O
    inst = I.ea_instance(L, index=gid)
    betas = I.geometric_betas(0.2, 3.0, R)
    o = O.Oracle(inst, betas, instance_id=gid, prop_enabled=[1] * (R - 1) + [0],
                 propose_every=5, seed=0x7A972509, pool_size=P)
    for r in range(R):
        o.load_pool(r, I.random_configs(inst.n_spins, P, seed=21, index=100 * gid + r))
    o.run_cycles(CYCLES)
    s, E, w = o.read()
    return s, E, w


def _rank_main(rank: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        ids = list(shard.weak_shard(rank, WORLD, PER_RANK))
        res = {gid: _run_instance(gid) for gid in ids}
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"),
                 ids=np.array(ids), **{f"s{g}": v[0] for g, v in res.items()},
                 **{f"E{g}": v[1] for g, v in res.items()}, **{f"w{g}": v[2] for g, v in res.items()})
        # ragged split computed independently on each rank
        costs = [Lk ** 3 * Rk for Lk, Rk in zip([6, 16, 8, 12, 10, 14, 6, 16, 8],
                                                 [24, 48, 30, 36, 40, 28, 33, 25, 47])]
        split = shard.balanced_shard(costs, WORLD)
        every = [None] * WORLD
        dist.all_gather_object(every, split)
        assert all(e == split for e in every)
        # max over ranks
        ms = shard.job_ms(10.0 + 5.0 * rank, dist, device=torch.device("cpu"))
        with open(os.path.join(out_dir, f"ms{rank}.txt"), "w") as f:
            f.write(repr(ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_reproduce_the_unsharded_run(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    seen = []
    for rank in range(WORLD):
        z = np.load(tmp_path / f"rank{rank}.npz")
        assert list(z["ids"]) == list(range(rank * PER_RANK, (rank + 1) * PER_RANK))
        for gid in z["ids"]:
            s, E, w = _run_instance(int(gid))          # the same instance, unsharded
            assert np.array_equal(z[f"s{gid}"], s)
            assert np.array_equal(z[f"E{gid}"], E)
            assert np.array_equal(z[f"w{gid}"], w)
            seen.append(int(gid))
        assert float((tmp_path / f"ms{rank}.txt").read_text()) == 15.0
    assert sorted(seen) == list(range(WORLD * PER_RANK))


def test_balanced_shard_is_a_partition_with_bounded_imbalance():
    g = np.random.default_rng(5)
    Ls = g.choice([6, 8, 10, 12, 14, 16], size=4096)
    Rs = g.integers(24, 49, size=4096)
    costs = (Ls.astype(np.int64) ** 3 * Rs).tolist()
    for world in (1, 2, 4, 8):
        parts = shard.balanced_shard(costs, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(4096))
        loads = [sum(costs[k] for k in p) for p in parts]
        # greedy LPT: the spread is at most the largest single cost
        assert max(loads) - min(loads) <= max(costs)


def test_weak_shard_and_rate():
    assert list(shard.weak_shard(1, 4, 256)) == list(range(256, 512))
    with pytest.raises(ValueError):
        shard.weak_shard(4, 4, 1)
    # 2 ranks x 1e6 units in 1 ms (1e6 ns) = 2 units per ns
    assert shard.job_rate(10 ** 6, 2, 1.0) == pytest.approx(2.0)
    assert shard.job_ms(3.5) == 3.5
