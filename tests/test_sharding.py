"""Sharding of the batched path over ranks: host logic on the CPU, and a
world-size-2 gloo run of the same code the benchmark uses under torchrun."""

import os
import socket

import numpy as np
import pytest

from paper_2401_13772_gb300.sharding import lpt_shards, max_over_ranks, shard_parts


def test_lpt_is_a_balanced_partition():
    rng = np.random.default_rng(0)
    n = 4 * rng.integers(16, 193, size=4000)
    for world in (1, 2, 3, 4, 8):
        shards = [shard_parts(n, world, r) for r in range(world)]
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(n)))  # every part exactly once
        loads = [float(np.sum(n[s].astype(np.float64) ** 3)) for s in shards]
        # greedy LPT: no rank exceeds the mean by more than the largest part
        assert max(loads) - sum(loads) / world <= float(n.max()) ** 3


def test_lpt_small_cases():
    assert lpt_shards([1.0, 1.0, 1.0], 2) == [[0, 2], [1]]
    assert lpt_shards([5.0, 1.0, 1.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3, 4, 5]]
    assert lpt_shards([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        lpt_shards([1.0], 0)
    with pytest.raises(ValueError):
        shard_parts([4, 8], 2, 2)


def test_without_process_group_values_pass_through():
    assert max_over_ranks(3.5) == 3.5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        mine = shard_parts(n, world, rank)
        # what the benchmark does: per-rank time, the maximum over ranks, and
        # the parts of all ranks
        t = 1.0 + rank
        tmax = max_over_ranks(t)
        import torch
        counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(counts, torch.tensor([len(mine)], dtype=torch.int64))
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([tmax, sum(int(c.item()) for c in counts)] + mine, dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding(tmp_path):
    import torch.multiprocessing as mp
    n = 4 * np.random.default_rng(1).integers(16, 193, size=300)
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, join=True)
    got = [np.load(os.path.join(tmp_path, f"r{r}.npy")) for r in range(world)]
    for g in got:
        assert g[0] == 2.0          # max of per-rank times 1.0 and 2.0
        assert int(g[1]) == len(n)  # the shards cover every part
    parts = sorted(int(i) for g in got for i in g[2:])
    assert parts == list(range(len(n)))
