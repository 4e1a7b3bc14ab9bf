"""The synthetic generator: normalisation, determinism and its pose convention.

The last test ties the generator's rendering convention (rotate by alpha,
shift by t, mirror) to the oracle's pose meaning: a noise-free particle is
recovered at s = Mm t and angle index (-alpha M / 2 pi) mod M.
"""
import math

import numpy as np
import torch

import synth
from oracle import mra_oracle as O


def test_refs_are_normalised_and_seeded():
    refs, blob = synth.make_refs(4, 40, blobs=10, sigma=(2.0, 4.0), disc=12.0, seed=5)
    assert refs.shape == (4, 40, 40)
    np.testing.assert_allclose(refs.mean(dim=(1, 2)).numpy(), 0.0, atol=1e-12)
    np.testing.assert_allclose(refs.std(dim=(1, 2), unbiased=False).numpy(), 1.0, atol=1e-12)
    refs2, _ = synth.make_refs(4, 40, blobs=10, sigma=(2.0, 4.0), disc=12.0, seed=5)
    assert torch.equal(refs, refs2)


def test_particles_normalised_and_truth_ranges():
    w = synth.WORKLOADS["mra_n500_L76_K10_shift2"]
    refs, imgs, truth, _ = synth.make_workload(w, n=64)
    assert imgs.shape == (64, 76, 76) and imgs.dtype == torch.float32
    np.testing.assert_allclose(imgs.double().mean(dim=(1, 2)).numpy(), 0.0, atol=1e-5)
    np.testing.assert_allclose(imgs.double().std(dim=(1, 2), unbiased=False).numpy(), 1.0, atol=1e-5)
    assert truth.k.min() >= 0 and truth.k.max() < 10
    assert np.abs(truth.t).max() <= 2
    assert set(np.unique(truth.m)) <= {0, 1}


def test_workload_shift_grids():
    assert len(synth.shift_grid(2.0, 1.0)) == 5
    assert len(synth.shift_grid(4.0, 1.0)) ** 2 == 81
    assert len(synth.shift_grid(6.0, 1.0)) ** 2 == 169


def test_generator_pose_convention_matches_oracle():
    L = 48
    refs, blob = synth.make_refs(2, L, blobs=8, sigma=(2.5, 4.0), disc=8.0, seed=11)
    cfg = O.MRAConfig(L, 2, 16, 1, 2.0, 1.0, 1)
    M = O.angle_count(O.ring_table(2, 16, 1))
    j0 = np.array([37, 90, 5])
    truth = synth.ParticleTruth(k=np.array([0, 1, 1]), alpha=2 * math.pi * j0 / M,
                                t=np.array([[1, -2], [-2, 0], [0, 2]]), m=np.array([0, 1, 1]))
    imgs = synth.render_particles(blob, truth, snr=None, normalise=False)
    spec = O.reference_spectra(refs.numpy(), cfg)
    for i in range(3):
        k = int(truth.k[i])
        c = O.cc_table(imgs[i].numpy(), spec, cfg)[k:k + 1]
        p = O._pose_from_table(c, cfg)
        tx, ty = truth.t[i]
        assert p.mirror == truth.m[i]
        assert p.ang_idx == (-j0[i]) % M
        assert (p.sx, p.sy) == (float(-tx if truth.m[i] else tx), float(ty))
