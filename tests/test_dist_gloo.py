"""Multi-process path on CPU (gloo, world size 2): channel-block sharding with
no data-path exchange reassembles the full integral, and the timing reduction
takes the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_34025_b300.dist import channel_block, tree_block


def test_channel_blocks_partition():
    for d in (0, 1, 7, 16, 64):
        for world in (1, 2, 3, 8):
            blocks = [channel_block(r, world, d) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == d
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    assert tree_block(1, 2, 4096) == (2048, 4096)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import workloads as W
    from oracle import brute
    from paper_2609_34025_b300.dist import max_over_ranks

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = W.configs.rrt_n2000(n=300, d=6)
    F = W.normal_field(300, 6, seed=123)
    c0, c1 = channel_block(rank, world, 6)
    part = brute.integrate(cfg["tree"], cfg["delta"], cfg["kernel"], F[:, c0:c1].astype(np.float64))
    np.save(os.path.join(out_dir, f"part{rank}.npy"), part)
    t = max_over_ranks(10.0 + rank)
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_shard_and_reduce(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    import workloads as W
    from oracle import brute

    cfg = W.configs.rrt_n2000(n=300, d=6)
    F = W.normal_field(300, 6, seed=123).astype(np.float64)
    full = brute.integrate(cfg["tree"], cfg["delta"], cfg["kernel"], F)
    got = np.concatenate([np.load(tmp_path / f"part{r}.npy") for r in range(2)], axis=1)
    np.testing.assert_allclose(got, full, rtol=1e-13, atol=1e-13)
    assert all(float(np.load(tmp_path / f"t{r}.npy")[0]) == 11.0 for r in range(2))
