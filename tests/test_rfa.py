"""Reference-free alignment (single common reference built from the data):
one pass against the oracle's pass, and recovery of the particles' relative
orientations on a clean stack."""
import math

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


def _stack(n, L, shift, mirror, snr, seed):
    _, blob = synth.make_refs(1, L, blobs=10, sigma=(0.05 * L, 0.1 * L), disc=0.22 * L, seed=seed)
    imgs, truth = synth.make_particles(blob, n, shift_range=shift, mirror=mirror, snr=snr, seed=seed + 1,
                                       noise_seed=seed + 2)
    return imgs.float().contiguous(), truth


def test_rfa_pass_matches_oracle(mra):
    from oracle import mra_oracle as O
    from paper_2011_05755_gb300.rfa import rfa, unaligned_mean
    imgs, _ = _stack(40, 32, 1, True, 1.0, 61)
    cfg = O.MRAConfig(32, 1, 12, 1, 1.0, 1.0, 1)
    imgs64 = imgs.double().numpy()
    dimgs = imgs.to(DEV)
    al = mra.Aligner(32, 1, 12, 1, 1.0, 1.0, 1)
    ref0 = unaligned_mean(al, dimgs)
    al.close()
    want0 = O.normalize(imgs64.mean(axis=0))
    np.testing.assert_allclose(ref0.cpu().double().numpy(), want0, atol=2e-5)

    out = rfa(dimgs, dict(L=32, first_ring=1, last_ring=12, ring_step=1, shift_range=1.0, shift_step=1.0, mirror=1),
              n_iter=1, ref0=ref0)
    got = mra.decode_poses(out["poses"])
    ref64 = ref0.cpu().double().numpy()[None]
    spec = O.reference_spectra(ref64, cfg)
    M = O.angle_count(O.ring_table(1, 12, 1))
    shifts = O.shift_list(1.0, 1.0)
    for i in range(len(imgs64)):
        table = O.cc_table(imgs64[i], spec, cfg)
        best = table.max()
        pick = table[0, got["shift_idx"][i], got["mirror"][i], got["ang_idx"][i]]
        assert pick >= best - 1e-4 * abs(best), (i, pick, best)
    # given the library's poses, the oracle's average, normalised, is the new reference
    poses = [O.Pose(0, int(s), int(m), int(j), shifts[int(s)][0], shifts[int(s)][1], 0.0, 0.0, 0.0)
             for s, m, j in zip(got["shift_idx"], got["mirror"], got["ang_idx"])]
    avg, counts = O.average(imgs64, poses, 1, M)
    assert counts[0] == len(imgs64)
    np.testing.assert_allclose(out["ref"].cpu().double().numpy(), O.normalize(avg[0]), atol=5e-5)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_rfa_recovers_relative_orientations(mra, prec):
    from paper_2011_05755_gb300.rfa import rfa
    imgs, truth = _stack(300, 48, 0, False, 2.0, 71)
    precision = mra.MRA_FP32 if prec == "fp32" else mra.MRA_BF16_RESCORE
    out = rfa(imgs.to(DEV), dict(L=48, first_ring=2, last_ring=18, ring_step=1, shift_range=1.0, shift_step=1.0,
                                 mirror=1), n_iter=8, tol=0.0, precision=precision)
    p = mra.decode_poses(out["poses"])
    from oracle import mra_oracle as O
    M = O.angle_count(O.ring_table(2, 18, 1))
    phi = 2 * math.pi * p["ang_idx"] / M
    # one mirror state for all, and the estimated angle differs from the true
    # one by a common rotation (sign depending on that mirror state)
    m = p["mirror"]
    assert max(np.mean(m == 0), np.mean(m == 1)) > 0.95
    conc = max(abs(np.mean(np.exp(1j * (phi + truth.alpha)))), abs(np.mean(np.exp(1j * (phi - truth.alpha)))))
    assert conc > 0.9, (conc, out["history"])
    ch = [h["changed"] for h in out["history"]]
    assert ch[-1] < 0.1, ch
