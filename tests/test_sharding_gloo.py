"""World-size-2 sharding of the class average on CPU ranks (gloo).

Each rank takes its contiguous shard, forms its class sums (here with the
oracle's aligned images, standing in for mra_class_sums, which needs a GPU),
the product's exchange step sums them over ranks, and the finalised average
must equal the unsharded oracle average.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2011_05755_gb300.shard import allreduce_class_sums, shard_range


def test_shard_range_partitions():
    for n in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            parts = [shard_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, imgs, poses, K, M, out):
    from oracle import mra_oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = shard_range(len(imgs), world, rank)
    L = imgs.shape[-1]
    sums = torch.zeros((K, L, L), dtype=torch.float64)
    comp = torch.zeros_like(sums)
    counts = torch.zeros((K,), dtype=torch.int64)
    for i in range(a, b):
        p = poses[i]
        sums[p.k] += torch.from_numpy(O.aligned_image(imgs[i], p.sx, p.sy, p.mirror, 2 * math.pi * p.ang_idx / M))
        counts[p.k] += 1
    allreduce_class_sums(sums, comp, counts)
    if rank == 0:
        out.put((sums.numpy(), comp.numpy(), counts.numpy()))
    dist.destroy_process_group()


def test_two_rank_class_average_matches_unsharded():
    from oracle import mra_oracle as O
    import synth
    L, K = 24, 3
    refs, blob = synth.make_refs(K, L, blobs=6, sigma=(1.5, 3.0), disc=5.0, seed=3)
    imgs, _ = synth.make_particles(blob, 11, shift_range=1, mirror=True, snr=2.0, seed=4, noise_seed=5)
    imgs = imgs.numpy()
    cfg = O.MRAConfig(L, 1, 8, 1, 1.0, 1.0, 1)
    M = O.angle_count(O.ring_table(1, 8, 1))
    poses = O.align(imgs, refs.numpy(), cfg)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, imgs, poses, K, M, q)) for r in range(2)]
    for p in procs:
        p.start()
    sums, comp, counts = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    avg_ref, cnt_ref = O.average(imgs, poses, K, M)
    assert np.array_equal(counts, cnt_ref)
    for k in range(K):
        if counts[k]:
            np.testing.assert_allclose((sums[k] + comp[k]) / counts[k], avg_ref[k], atol=1e-12)
