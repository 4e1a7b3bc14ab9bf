"""The no-allocation entry point mra_align_static against mra_align.

mra_align_static serves callers that may not allocate device memory: it
takes no handle and keeps all its intermediates in one array the library
reserves at load time.  Its poses must equal those of the handle-based
mra_align (the same kernels run in the same order per image), on two calls
in a row, the second one reusing the array the first one left behind.  The
stack is large enough that the array holds it only in several chunks.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
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


def test_static_scratch_alignment_matches_handle_path(mra):
    L, r1, r2, R = 76, 1, 35, 2.0
    refs, blob = synth.make_refs(10, L, seed=1201)
    imgs, _ = synth.make_particles(blob, 150, shift_range=2, mirror=True, snr=0.1, seed=1202, noise_seed=1203)
    refs = refs.float().contiguous().to(DEV)
    imgs = imgs.float().contiguous().to(DEV)

    al = mra.Aligner(L, r1, r2, 1, R, 1.0, 1, mra.MRA_FP32)
    al.set_refs(refs)
    want = mra.decode_poses(al.align(imgs))
    al.close()

    for call in range(2):
        out = torch.full((imgs.shape[0], 8), -1, dtype=torch.int32, device=DEV)
        mra.mra_align_static(refs, imgs, out, L, r1, r2, 1, R, 1.0, 1)
        got = mra.decode_poses(out)
        for key in ("k", "ang_idx", "mirror", "shift_idx"):
            assert np.array_equal(got[key], want[key]), (call, key)
        np.testing.assert_allclose(got["cc"], want["cc"], rtol=1e-4, atol=0)


def test_static_scratch_rejects_oversized_configuration(mra):
    refs = torch.zeros((4000, 128, 128), dtype=torch.float32, device=DEV)
    imgs = torch.zeros((1, 128, 128), dtype=torch.float32, device=DEV)
    out = torch.empty((1, 8), dtype=torch.int32, device=DEV)
    with pytest.raises(mra.MRAError) as ei:
        mra.mra_align_static(refs, imgs, out, 128, 1, 60, 1, 6.0, 1.0, 1)
    assert ei.value.code == mra.MRA_EINVAL
    assert "bytes" in str(ei.value)
