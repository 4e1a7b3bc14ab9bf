"""The whole pass as one CUDA graph (mra_run_graph) against the eager calls.

mra_run_graph runs set_refs + align + class average eagerly on the first
call with a set of buffers, captures them on the second and replays the
graph afterwards.  The replayed graph must give bit-identical poses, counts
and averages to the eager per-chunk launches, also after the buffers'
contents change, and a call with other buffers must start again.
"""
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mra():
    import __graft_entry__ as entry
    entry.build()
    import paper_2011_05755_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    return m


def _stack(L, K, n, seed):
    refs, blob = synth.make_refs(K, L, blobs=10, sigma=(L / 20, L / 10), disc=L / 4, seed=seed)
    imgs, _ = synth.make_particles(blob, n, shift_range=2, mirror=True, snr=0.5, seed=seed + 1, noise_seed=seed + 2)
    return refs.float().contiguous().to(DEV), imgs.float().contiguous().to(DEV)


@pytest.mark.parametrize("precision,kernel", [(0, 0), (1, 1), (1, 2)])
def test_graph_pass_equals_eager_calls(mra, precision, kernel):
    L, K, n = 76, 11, 700
    refs, imgs = _stack(L, K, n, seed=61)
    # several chunks and a ragged tail
    al = mra.Aligner(L, 1, 35, 1, 2.0, 1.0, 1, precision, chunk_images=256, kernel=kernel)
    al.set_refs(refs)
    want_p = al.align(imgs)
    want_a, want_c = al.average(imgs, want_p)
    torch.cuda.synchronize()
    g = mra.Aligner(L, 1, 35, 1, 2.0, 1.0, 1, precision, chunk_images=256, kernel=kernel)
    poses = torch.zeros((n, 8), dtype=torch.int32, device=DEV)
    avg = torch.zeros((K, L, L), device=DEV)
    cnt = torch.zeros((K,), dtype=torch.int32, device=DEV)
    for call in range(4):
        poses.zero_()
        avg.zero_()
        mra.mra_run_graph(g.h, refs, imgs, poses, avg, cnt)
        torch.cuda.synchronize()
        assert mra.mra_graph_info(g.h) == (call >= 1)
        assert torch.equal(poses, want_p), call
        assert torch.equal(cnt, want_c), call
        assert torch.equal(avg, want_a), call
    # new contents in the same buffers: the replayed graph reads them
    refs2, imgs2 = _stack(L, K, n, seed=71)
    refs.copy_(refs2)
    imgs.copy_(imgs2)
    al.set_refs(refs)
    want_p = al.align(imgs)
    want_a, want_c = al.average(imgs, want_p)
    mra.mra_run_graph(g.h, refs, imgs, poses, avg, cnt)
    torch.cuda.synchronize()
    assert mra.mra_graph_info(g.h)
    assert torch.equal(poses, want_p) and torch.equal(cnt, want_c) and torch.equal(avg, want_a)
    # other buffers: the graph is dropped and the pass runs eagerly again
    imgs3 = imgs[: n - 50].clone()
    poses3 = torch.zeros((n - 50, 8), dtype=torch.int32, device=DEV)
    mra.mra_run_graph(g.h, refs, imgs3, poses3, avg, cnt)
    torch.cuda.synchronize()
    assert not mra.mra_graph_info(g.h)
    assert torch.equal(poses3, want_p[: n - 50])
    al.close()
    g.close()


def test_autotune_picks_the_fastest_candidate_and_caches_it(mra, tmp_path):
    from paper_2011_05755_gb300.autotune import tune, tuned_aligner
    cache = str(tmp_path / "tune.json")
    a = tune(76, 1, 35, 1, 1.0, 1.0, 1, mra.MRA_BF16_RESCORE, 16, n_probe=512, cache=cache)
    kinds = {c["kernel"] for c in a["candidates"]}
    assert kinds == {mra.MRA_KERNEL_MMA_SYNC, mra.MRA_KERNEL_TCGEN05}
    assert a["ms_per_image"] == min(c["ms_per_image"] for c in a["candidates"])
    assert (a["kernel"], a["chunk_images"]) in {(c["kernel"], c["chunk_images"]) for c in a["candidates"]}
    b = tune(76, 1, 35, 1, 1.0, 1.0, 1, mra.MRA_BF16_RESCORE, 16, n_probe=512, cache=cache)
    assert b == a  # from the cache
    al, choice = tuned_aligner(76, 1, 35, 1, 1.0, 1.0, 1, mra.MRA_BF16_RESCORE, 16, n_probe=512, cache=cache)
    assert choice == a
    al.close()
