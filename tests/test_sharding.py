"""Sharding across ranks (CPU, gloo, world size 2): split the grasps, run
the FP64 oracle's coarse-stage loop on each shard, gather -- the result is
bitwise equal to the unsharded run (grasps are independent)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2412_16490_gb300.sharding import gather_shards, shard_range


def test_shard_ranges_partition_the_batch():
    for B in (0, 1, 7, 64, 4097):
        for world in (1, 2, 3, 8):
            spans = [shard_range(B, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == B
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def _worker(rank, world, port, B, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bodex_inputs as I
    import oracle as O
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=B)
    lo, hi = shard_range(B, rank, world)
    x, _, _, E = O.run(O.Hand(hand), O.Object(obj), x0[lo:hi], T, P, n_steps=3, grad_mode="analytic", threads=1)
    full = gather_shards(torch.from_numpy(np.concatenate([x, E[:, None]], 1)), B, dist)
    if rank == 0:
        np.save(out_path, full.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_run_equals_unsharded(tmp_path):
    import bodex_inputs as I
    import oracle as O
    O.build()
    B = 11
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, port, B, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=B)
    x, _, _, E = O.run(O.Hand(hand), O.Object(obj), x0, T, P, n_steps=3, grad_mode="analytic", threads=1)
    assert np.array_equal(got, np.concatenate([x, E[:, None]], 1))
