"""World-size-2 sharding of the class average (gloo).

The CPU test covers the partition and the exchange step: each rank takes its
contiguous shard, forms its class sums with the oracle's aligned images (a
stand-in for mra_class_sums, which needs a GPU), the product's exchange step
sums them over ranks, and the finalised average must equal the unsharded
oracle average.  The GPU test covers the library's half: the ranks form
their sums with mra_class_sums and finalise with mra_average_finalize.
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


def _gpu_worker(rank, world, port, imgs, refs, poses, cfg, K, out):
    """One rank: its shard's compensated class sums through the library (mra_class_sums on the GPU),
    the exchange step over gloo on host copies, and the finalised average (mra_average_finalize)."""
    import paper_2011_05755_gb300 as mra
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    a, b = shard_range(len(imgs), world, rank)
    L = imgs.shape[-1]
    al = mra.Aligner(*cfg)
    al.set_refs(refs.cuda())  # the class sums need the handle's K
    sums = torch.zeros((K, L, L), device="cuda")
    comp = torch.zeros_like(sums)
    counts = torch.zeros((K,), dtype=torch.int32, device="cuda")
    if b > a:
        mra.mra_class_sums(al.h, imgs[a:b].cuda().contiguous(), torch.from_numpy(poses[a:b]).cuda().contiguous(),
                           sums, comp, counts)
    hs, hc, hn = sums.cpu(), comp.cpu(), counts.cpu()
    allreduce_class_sums(hs, hc, hn)
    avg = torch.zeros((K, L, L), device="cuda")
    mra.mra_average_finalize(al.h, hs.cuda(), hc.cuda(), hn.cuda(), avg)
    if rank == 0:
        out.put((avg.cpu().numpy(), hn.numpy()))
    al.close()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_rank_library_class_sums_match_unsharded_average():
    """The library's half of the exchange: two ranks (processes on the one GPU, whose kernels never wait
    on each other) form their shards' sums with mra_class_sums, all-reduce them over gloo and finalise;
    the result equals mra_average of the whole stack within FP32 rounding."""
    import paper_2011_05755_gb300 as mra
    import synth
    import __graft_entry__ as entry
    entry.build()
    L, K = 40, 5
    refs, blob = synth.make_refs(K, L, blobs=8, sigma=(2.0, 4.0), disc=8.0, seed=13)
    imgs, _ = synth.make_particles(blob, 301, shift_range=2, mirror=True, snr=1.0, seed=14, noise_seed=15)
    imgs = imgs.float().contiguous()
    cfg = (L, 1, 16, 1, 2.0, 1.0, 1)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    # poses and the unsharded average in a child too: this process never initialises CUDA
    procs = [ctx.Process(target=_unsharded_worker, args=(imgs, refs.float().contiguous(), cfg, q))]
    procs[0].start()
    poses, want_avg, want_cnt = q.get(timeout=300)
    procs[0].join(timeout=60)
    assert procs[0].exitcode == 0
    port = _free_port()
    procs = [ctx.Process(target=_gpu_worker, args=(r, 2, port, imgs, refs.float().contiguous(), poses, cfg, K, q))
             for r in range(2)]
    for p in procs:
        p.start()
    avg, cnt = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.array_equal(cnt, want_cnt)
    np.testing.assert_allclose(avg, want_avg, rtol=0, atol=1e-5)


def _unsharded_worker(imgs, refs, cfg, out):
    import paper_2011_05755_gb300 as mra
    torch.cuda.set_device(0)
    al = mra.Aligner(*cfg)
    al.set_refs(refs.cuda())
    poses = al.align(imgs.cuda())
    avg, cnt = al.average(imgs.cuda(), poses)
    # NumPy arrays travel by value: a tensor would travel as a file descriptor that can vanish when
    # this process exits before the parent has received it
    out.put((poses.cpu().numpy(), avg.cpu().numpy(), cnt.cpu().numpy()))
    al.close()
