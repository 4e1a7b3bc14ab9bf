"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP32 path): every CC value within 1e-4 of the Cauchy-Schwarz
scale sqrt(E_x E_y) of its row, E = sum_r dr r (2 pi / N_r) sum_q v_q^2;
the best CC within 1e-4 relative; the pose (k, shift, mirror, angle)
identical whenever the oracle's best beats its runner-up by more than 1e-3
relative (otherwise the GPU's pose must score within tolerance of the best);
class averages within 1e-4 relative L2 given the oracle's poses.  Ring
samples and spectra are compared at FP32 rounding scale.
"""
import os
import zlib

import numpy as np
import pytest
import torch

import synth
from oracle import mra_oracle as O
from oracle_pool import oracle_poses, table_value

pytestmark = pytest.mark.gpu

CC_TOL = 1e-4
GAP = 1e-3


@pytest.fixture(scope="module")
def mra():
    import __graft_entry__ as entry
    entry.build()
    import paper_2011_05755_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    return m


DEV = "cuda:0"

CASES = {
    # name: (L, r1, r2, dr, R, step, mirror, K, n)
    "M128_ragged": (32, 1, 12, 1, 1.5, 0.5, 1, 11, 5),
    "M128_step2_nomirror": (48, 2, 20, 2, 2.0, 1.0, 0, 3, 4),
    "M128_outside_box": (24, 1, 15, 1, 2.0, 1.0, 1, 2, 3),
    "M256_L76": (76, 1, 35, 1, 2.0, 1.0, 1, 10, 4),
    "M512_L128": (128, 1, 60, 1, 1.0, 1.0, 1, 3, 2),
    "M16": (16, 1, 2, 1, 1.0, 1.0, 1, 2, 3),
    "M32": (16, 1, 4, 1, 1.0, 1.0, 1, 2, 3),
    "M64": (20, 1, 6, 1, 2.0, 1.0, 1, 9, 3),
    # M = 256 with sparse rings (3, 6, ..., 24: other R_f and frequency groups) and K not a tile multiple
    "M256_r24_step": (56, 3, 24, 3, 1.0, 1.0, 1, 13, 3),
    "M256_nomirror": (64, 2, 30, 1, 2.0, 1.0, 0, 9, 3),
    # rings beyond 64 at L = 132 (the 16-bit paths' FP32 rescore keeps each ring's spectrum in its samples)
    "M512_r65": (132, 1, 65, 1, 1.0, 1.0, 1, 3, 2),
    # a box whose rows are not a multiple of 16 bytes: the polar kernel stages the image with plain loads
    # instead of the TMA tensor copy
    "M128_L30": (30, 1, 12, 1, 2.0, 1.0, 1, 5, 3),
}


def _inputs(L, K, n, R, mirror, seed):
    refs, blob = synth.make_refs(K, L, blobs=10, sigma=(max(1.5, L / 20), max(2.5, L / 10)), disc=L / 4, seed=seed)
    imgs, _ = synth.make_particles(blob, n, shift_range=int(R), mirror=bool(mirror), snr=1.0, seed=seed + 1,
                                   noise_seed=seed + 2)
    return refs.float().contiguous(), imgs.float().contiguous()


def _oracle_table(imgs, refs, cfg):
    spec = O.reference_spectra(refs.double().numpy(), cfg)
    return np.stack([O.cc_table(im.double().numpy(), spec, cfg) for im in imgs])


def _cs_scale(imgs, refs, cfg):
    """sqrt(E_x E_y) per (image, k, s, m)."""
    rings = O.ring_table(cfg.first_ring, cfg.last_ring, cfg.ring_step)
    w = O.ring_weights(rings, cfg.ring_step)
    ey = np.array([sum(wi * np.dot(y, y) for wi, y in zip(w, O.polar_samples(r.double().numpy(), rings)))
                   for r in refs])
    mirrors = (0, 1) if cfg.mirror else (0,)
    out = []
    for im in imgs:
        ex = np.array([[sum(wi * np.dot(x, x) for wi, x in zip(w, O.polar_samples(im.double().numpy(), rings, sx,
                                                                                    sy, m)))
                        for m in mirrors] for sx, sy in O.shift_list(cfg.shift_range, cfg.shift_step)])
        out.append(np.sqrt(ey[:, None, None] * ex[None, :, :]))
    return np.stack(out)


@pytest.mark.parametrize("name", list(CASES))
def test_stage_parity(mra, name):
    L, r1, r2, dr, R, step, mirror, K, n = CASES[name]
    refs, imgs = _inputs(L, K, n, R, mirror, seed=zlib.crc32(name.encode()) % 1000)
    cfg = O.MRAConfig(L, r1, r2, dr, R, step, mirror)
    rings = O.ring_table(r1, r2, dr)
    M = O.angle_count(rings)
    al = mra.Aligner(L, r1, r2, dr, R, step, mirror, mra.MRA_FP32)
    dimgs = imgs.to(DEV)
    al.set_refs(refs.to(DEV))
    samples = al.debug_polar(dimgs).cpu().numpy()
    spectra = al.debug_spectra(dimgs).cpu().numpy()
    table = al.debug_cc(dimgs).cpu().numpy()
    torch.cuda.synchronize()
    shifts = O.shift_list(R, step)
    # (1) ring samples and (2) ring spectra, unmirrored, every shift.
    # Sample tolerance from the FP32 arithmetic: the sample position
    # c0 + s + r (cos, sin) is rounded to ~L 2^-24 in each coordinate, and a
    # bilinear sample moves by at most 2 max|I| per pixel of displacement,
    # plus a few ulps of the interpolation itself.
    for i in range(n):
        im = imgs[i].double().numpy()
        amax = float(np.abs(im).max())
        s_tol = 4.0 * amax * L * 2.0 ** -24 + 8.0 * amax * 2.0 ** -24
        for si, (sx, sy) in enumerate(shifts):
            xs = O.polar_samples(im, rings, sx, sy, 0)
            np.testing.assert_allclose(samples[i, si], np.concatenate(xs), atol=s_tol, rtol=0)
            # Spectra: |DFT(dx)(f)| <= ||dx||_1 for the sample differences dx,
            # plus FFT rounding ~ log2(N) 2^-24 sqrt(N) ||x|| per bin.
            got = spectra[i, si, :, 0] + 1j * spectra[i, si, :, 1]
            off_s = 0
            off_b = 0
            for x in xs:
                N = len(x)
                ref = O.ring_dft(x)[N // 2:]
                g = got[off_b:off_b + N // 2 + 1]
                l1 = float(np.abs(samples[i, si, off_s:off_s + N] - x).sum())
                tol = l1 + 4.0 * np.log2(N) * 2.0 ** -24 * np.sqrt(N) * np.linalg.norm(x) + 1e-12
                assert np.max(np.abs(g - ref)) <= tol, (i, si, N, float(np.max(np.abs(g - ref))), tol)
                off_s += N
                off_b += N // 2 + 1
    # (3) the full CC table
    ot = _oracle_table(imgs, refs, cfg)                     # [n, K, S, m, M]
    scale = _cs_scale(imgs, refs, cfg)                      # [n, K, S, m]
    got = table if mirror else table[:, :, :, :1, :]
    err = np.abs(got - ot) / scale[..., None]
    assert err.max() <= CC_TOL, (name, float(err.max()))


# 16-bit contraction tolerance on the CC table, from operand rounding with
# unit roundoff u (BF16: 8 significant bits, u = 2^-8; FP16: 11, u = 2^-11):
# each product q v carries at most 2 u relative error; summed over (f, r) and
# bounded by Cauchy-Schwarz against the Parseval energies this is
# <= 8 u sqrt(E_x E_y) per angle.  For M = 256 the inverse angular DFT also
# runs on tensor cores with BF16 operands: the spectrum, the two DFT matrices
# and the twiddled intermediate are each rounded once, at most
# 4 * 2^-8 sqrt(E_x E_y) more.
def tc_tol(prec, M):
    # 8 unit roundoffs of the contraction operands; for M >= 256 the angular
    # spectrum (and, at M = 512, the inverse DFT's intermediate) is held in
    # BF16, each rounding bounded by 2^-9 of the Cauchy-Schwarz scale
    u = 2.0 ** -8 if prec == "bf16" else 2.0 ** -11
    return 8 * u + (4 * 2.0 ** -8 if M >= 256 else 0.0)


KERNEL_CODE = {"default": 0, "mma_sync": 1, "tcgen05": 2}
TC_CASES = [(name, "default") for name in ["M128_ragged", "M128_step2_nomirror", "M512_L128", "M512_r65", "M16",
                                             "M64"]] + \
    [("M256_L76", "mma_sync"), ("M256_L76", "tcgen05"), ("M256_r24_step", "tcgen05"), ("M256_nomirror", "tcgen05")]


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("name,kernel", TC_CASES)
def test_stage_parity_tensor_core(mra, name, kernel, prec):
    """The CC table from the 16-bit tensor-core contraction (before rescoring) against the oracle."""
    L, r1, r2, dr, R, step, mirror, K, n = CASES[name]
    refs, imgs = _inputs(L, K, n, R, mirror, seed=zlib.crc32(name.encode()) % 1000)
    cfg = O.MRAConfig(L, r1, r2, dr, R, step, mirror)
    precision = mra.MRA_BF16_RESCORE if prec == "bf16" else mra.MRA_FP16_RESCORE
    al = mra.Aligner(L, r1, r2, dr, R, step, mirror, precision, kernel=KERNEL_CODE[kernel])
    al.set_refs(refs.to(DEV))
    table = al.debug_cc(imgs.to(DEV)).cpu().numpy()
    ot = _oracle_table(imgs, refs, cfg)
    scale = _cs_scale(imgs, refs, cfg)
    got = table if mirror else table[:, :, :, :1, :]
    err = np.abs(got - ot) / scale[..., None]
    M = O.angle_count(O.ring_table(r1, r2, dr))
    assert err.max() <= tc_tol(prec, M), (name, prec, float(err.max()))
    print(name, prec, "max error / bound", float(err.max()) / tc_tol(prec, M))
    al.close()


POSE_CASES = [(name, prec, "default") for name in CASES for prec in ("fp32", "bf16", "fp16")] + \
    [(name, prec, "tcgen05") for name in ("M256_L76", "M256_r24_step", "M256_nomirror") for prec in ("bf16", "fp16")]


@pytest.mark.parametrize("name,prec,kernel", POSE_CASES)
def test_pose_and_average_parity(mra, name, prec, kernel):
    L, r1, r2, dr, R, step, mirror, K, n = CASES[name]
    refs, imgs = _inputs(L, K, n + 6, R, mirror, seed=7 + zlib.crc32(name.encode()) % 1000)
    precision = {"fp32": mra.MRA_FP32, "bf16": mra.MRA_BF16_RESCORE, "fp16": mra.MRA_FP16_RESCORE}[prec]
    _check_poses_and_averages(mra, refs, imgs, O.MRAConfig(L, r1, r2, dr, R, step, mirror), precision=precision,
                              kernel=KERNEL_CODE[kernel])


def _pose_rows(poses):
    rows = np.zeros((len(poses), 8), dtype=np.int32)
    fl = rows.view(np.float32)
    for i, p in enumerate(poses):
        rows[i, :4] = (p.k, p.ang_idx, p.mirror, p.shift_idx)
        fl[i, 4:] = (p.angle_deg, p.sx, p.sy, p.cc)
    return rows


def _check_poses_and_averages(mra, refs, imgs, cfg, sample=None, precision=None, chunk_images=0, kernel=0):
    K = refs.shape[0]
    rings = O.ring_table(cfg.first_ring, cfg.last_ring, cfg.ring_step)
    M = O.angle_count(rings)
    al = mra.Aligner(cfg.L, cfg.first_ring, cfg.last_ring, cfg.ring_step, cfg.shift_range, cfg.shift_step,
                     cfg.mirror, mra.MRA_FP32 if precision is None else precision, chunk_images, kernel)
    dimgs = imgs.to(DEV) if not imgs.is_cuda else imgs
    al.set_refs(refs.to(DEV))
    gp = mra.decode_poses(al.align(dimgs))
    idx = range(imgs.shape[0]) if sample is None else sample
    spec = O.reference_spectra(refs.double().cpu().numpy(), cfg)
    ops = []
    for i in idx:
        im = imgs[i].double().cpu().numpy()
        tab = O.cc_table(im, spec, cfg)
        p = O._pose_from_table(tab, cfg)
        ops.append(p)
        assert abs(gp["cc"][i] - p.cc) <= CC_TOL * abs(p.cc), (i, gp["cc"][i], p.cc)
        got = (int(gp["k"][i]), int(gp["shift_idx"][i]), int(gp["mirror"][i]), int(gp["ang_idx"][i]))
        if p.rel_gap > GAP:
            assert got == (p.k, p.shift_idx, p.mirror, p.ang_idx), (i, got, p)
        else:  # near tie: the GPU's choice must be (numerically) optimal too
            assert tab[got[0], got[1], got[2], got[3]] >= p.cc - CC_TOL * abs(p.cc)
        sx, sy = O.shift_list(cfg.shift_range, cfg.shift_step)[got[1]]
        assert (gp["sx"][i], gp["sy"][i]) == (np.float32(sx), np.float32(sy))
        assert gp["angle_deg"][i] == pytest.approx(360.0 * got[3] / M, rel=1e-6)
    # class averages from the oracle's poses (identical poses on both sides)
    if sample is None:
        rows = torch.from_numpy(_pose_rows(ops)).to(DEV)
        avg, cnt = al.average(dimgs, rows)
        oavg, ocnt = O.average(imgs.double().cpu().numpy(), ops, K, M)
        assert np.array_equal(cnt.cpu().numpy(), ocnt)
        a = avg.double().cpu().numpy()
        for k in range(K):
            if ocnt[k]:
                e = np.linalg.norm(a[k] - oavg[k]) / np.linalg.norm(oavg[k])
                assert e <= 1e-4, (k, e)
            else:
                assert np.all(a[k] == 0.0)  # untouched (zero-initialised by Aligner.average)
    al.close()
    return gp


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_workload_n500_L76_K10(mra, prec):
    """The 500-image, K = 10, 25-shift workload, every image against the oracle."""
    w = synth.WORKLOADS["mra_n500_L76_K10_shift2"]
    refs, imgs, truth, _ = synth.make_workload(w)
    cfg = O.MRAConfig(w.L, w.first_ring, w.last_ring, w.ring_step, w.shift_range, w.shift_step, w.mirror)
    precision = mra.MRA_FP32 if prec == "fp32" else mra.MRA_BF16_RESCORE
    gp = _check_poses_and_averages(mra, refs, imgs, cfg, precision=precision)
    # at SNR 0.1 most particles still find their generating class
    assert np.mean(gp["k"] == truth.k) > 0.5


def _check_sampled(gp, sample, ops, where):
    """Poses of the sampled images against the oracle (tolerances of the module docstring); a pose
    that differs from the oracle's must be a near tie scoring within the tolerance of the best."""
    ties = 0
    for i, o in zip(sample, ops):
        assert abs(gp["cc"][i] - o["cc"]) <= CC_TOL * abs(o["cc"]), (where, i, gp["cc"][i], o["cc"])
        got = (int(gp["k"][i]), int(gp["shift_idx"][i]), int(gp["mirror"][i]), int(gp["ang_idx"][i]))
        want = (o["k"], o["shift_idx"], o["mirror"], o["ang_idx"])
        if o["rel_gap"] > GAP:
            assert got == want, (where, i, got, want, o["rel_gap"])
        elif got != want:
            v = table_value(o, got)
            assert v is not None and v >= o["cc"] - CC_TOL * abs(o["cc"]), (where, i, got, want, v, o["cc"])
            ties += 1
    return ties


@pytest.fixture(scope="module")
def n100k_case():
    """The 100,000-image, K = 100, 81-shift benchmark stack on the device and the oracle's poses for
    200 seeded images of it (computed once, in a spawn pool on the host cores)."""
    w = synth.WORKLOADS["mra_n100k_L76_K100_shift4"]
    refs, imgs, truth, _ = synth.make_workload(w, device=DEV)
    cfgd = dict(L=w.L, first_ring=w.first_ring, last_ring=w.last_ring, ring_step=w.ring_step,
                shift_range=w.shift_range, shift_step=w.shift_step, mirror=w.mirror)
    rng = np.random.default_rng(2024)
    sample = sorted(set(rng.choice(w.n, size=198, replace=False).tolist()) | {0, w.n - 1})
    ops = oracle_poses(imgs[sample].double().cpu().numpy(), refs.double().cpu().numpy(), cfgd)
    return w, refs, imgs, sample, ops


@pytest.mark.parametrize("prec,kernel", [("fp32", "default"), ("bf16", "mma_sync"), ("bf16", "tcgen05"),
                                         ("fp16", "tcgen05")])
def test_workload_n100k_L76_K100_sampled(mra, n100k_case, prec, kernel):
    """Full-size 100,000-image, K = 100, 81-shift stack in the benchmark's launch configuration;
    200 seeded images (first and last included) against the oracle."""
    w, refs, imgs, sample, ops = n100k_case
    precision = {"fp32": mra.MRA_FP32, "bf16": mra.MRA_BF16_RESCORE, "fp16": mra.MRA_FP16_RESCORE}[prec]
    al = mra.Aligner(w.L, w.first_ring, w.last_ring, w.ring_step, w.shift_range, w.shift_step, w.mirror, precision,
                     kernel=KERNEL_CODE[kernel])
    al.set_refs(refs)
    gp = mra.decode_poses(al.align(imgs))
    al.close()
    assert len(sample) == 200
    ties = _check_sampled(gp, sample, ops, (prec, kernel))
    assert ties <= len(sample) // 10, ties


@pytest.fixture(scope="module")
def l128_case():
    """The larger-box workload (L = 128, K = 200, rings 1..60, M = 512, 169 shifts): 600 images
    (several chunks and a ragged tail) and the oracle's poses for 64 seeded images of them."""
    w = synth.WORKLOADS["mra_n50k_L128_K200_shift6"]
    refs, imgs, _, _ = synth.make_workload(w, n=600)
    cfgd = dict(L=w.L, first_ring=w.first_ring, last_ring=w.last_ring, ring_step=w.ring_step,
                shift_range=w.shift_range, shift_step=w.shift_step, mirror=w.mirror)
    rng = np.random.default_rng(128)
    sample = sorted(set(rng.choice(600, size=62, replace=False).tolist()) | {0, 599})
    ops = oracle_poses(imgs[sample].double().numpy(), refs.double().numpy(), cfgd)
    return w, refs, imgs, sample, ops


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_workload_L128_K200_sampled(mra, l128_case, prec):
    w, refs, imgs, sample, ops = l128_case
    precision = {"fp32": mra.MRA_FP32, "bf16": mra.MRA_BF16_RESCORE, "fp16": mra.MRA_FP16_RESCORE}[prec]
    al = mra.Aligner(w.L, w.first_ring, w.last_ring, w.ring_step, w.shift_range, w.shift_step, w.mirror, precision)
    al.set_refs(refs.to(DEV))
    gp = mra.decode_poses(al.align(imgs.to(DEV)))
    al.close()
    assert len(sample) == 64
    ties = _check_sampled(gp, sample, ops, prec)
    assert ties <= len(sample) // 10, ties


def test_chunking_and_ragged_tail_match_single_chunk(mra):
    refs, imgs = _inputs(32, 9, 23, 1.0, 1, seed=77)
    outs = []
    for chunk in (0, 4, 7):
        al = mra.Aligner(32, 1, 12, 1, 1.0, 1.0, 1, mra.MRA_FP32, chunk)
        al.set_refs(refs.to(DEV))
        outs.append(al.align(imgs.to(DEV)).cpu())
        al.close()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_empty_and_single_image(mra):
    refs, imgs = _inputs(32, 3, 1, 1.0, 1, seed=5)
    al = mra.Aligner(32, 1, 10, 1, 1.0, 1.0, 1)
    al.set_refs(refs.to(DEV))
    empty = torch.empty((0, 32, 32), dtype=torch.float32, device=DEV)
    p0 = al.align(empty)
    assert p0.shape == (0, 8)
    avg = torch.full((3, 32, 32), 7.0, device=DEV)
    cnt = torch.full((3,), 9, dtype=torch.int32, device=DEV)
    al.average(empty, p0, avg, cnt)
    assert torch.all(cnt == 0) and torch.all(avg == 7.0)
    gp = _check_poses_and_averages(mra, refs, imgs, O.MRAConfig(32, 1, 10, 1, 1.0, 1.0, 1))
    assert len(gp["k"]) == 1
    al.close()


def test_average_is_deterministic_and_sharding_matches(mra):
    refs, imgs = _inputs(40, 5, 300, 2.0, 1, seed=11)
    al = mra.Aligner(40, 1, 16, 1, 2.0, 1.0, 1)
    dimgs = imgs.to(DEV)
    al.set_refs(refs.to(DEV))
    poses = al.align(dimgs)
    a1, c1 = al.average(dimgs, poses)
    a2, c2 = al.average(dimgs, poses)
    assert torch.equal(a1, a2) and torch.equal(c1, c2)
    # two shards summed on the host side of the exchange, then finalised
    sums = torch.zeros((5, 40, 40), device=DEV)
    comp = torch.zeros_like(sums)
    cnts = torch.zeros((5,), dtype=torch.int32, device=DEV)
    for a, b in ((0, 170), (170, 300)):
        mra.mra_class_sums(al.h, dimgs[a:b].contiguous(), poses[a:b].contiguous(), sums, comp, cnts)
    avg = torch.zeros_like(sums)
    mra.mra_average_finalize(al.h, sums, comp, cnts, avg)
    assert torch.equal(cnts, c1)
    assert torch.allclose(avg, a1, rtol=0, atol=1e-5)
    al.close()


def test_host_buffer_path_matches_device_path(mra):
    refs, imgs = _inputs(32, 4, 40, 1.0, 1, seed=21)
    al = mra.Aligner(32, 1, 12, 1, 1.0, 1.0, 1, mra.MRA_FP32, 16)
    al.set_refs(refs.to(DEV))
    dp = al.align(imgs.to(DEV))
    da, dc = al.average(imgs.to(DEV), dp)
    hp = torch.zeros((40, 8), dtype=torch.int32).pin_memory()
    ha = torch.zeros((4, 32, 32), dtype=torch.float32).pin_memory()
    hc = torch.zeros((4,), dtype=torch.int32).pin_memory()
    mra.mra_run_host(al.h, refs.pin_memory(), imgs.pin_memory(), hp, ha, hc)
    assert torch.equal(hp, dp.cpu())
    assert torch.equal(hc, dc.cpu())
    assert torch.equal(ha, da.cpu())
    al.close()


def test_status_codes_and_fault_injection(mra):
    refs, imgs = _inputs(32, 2, 3, 1.0, 1, seed=3)
    al = mra.Aligner(32, 1, 10, 1, 1.0, 1.0, 1)
    with pytest.raises(mra.MRAError) as ei:
        al.align(imgs.to(DEV))
    assert ei.value.code == mra.MRA_ESTATE
    with pytest.raises(mra.MRAError) as ei:
        mra.mra_create(32, 1, 200)          # M = 2048 > 512
    assert ei.value.code == mra.MRA_EINVAL
    al.set_refs(refs.to(DEV))
    for what, code in (("timeout", mra.MRA_ETIMEOUT), ("launch", mra.MRA_ECUDA)):
        os.environ["MRA_FAULT"] = what
        try:
            with pytest.raises(mra.MRAError) as ei:
                al.align(imgs.to(DEV))
            assert ei.value.code == code
        finally:
            del os.environ["MRA_FAULT"]
    # the handle stays usable after injected failures
    p = mra.decode_poses(al.align(imgs.to(DEV)))
    assert len(p["k"]) == 3
    al.close()


@pytest.mark.parametrize("prec,L,r2,kernel", [("fp32", 32, 12, 0), ("bf16", 32, 12, 0), ("bf16", 76, 35, 1),
                                               ("bf16", 76, 35, 2)])
def test_device_wait_timeout_is_reported_and_recoverable(mra, prec, L, r2, kernel):
    """A bounded mbarrier wait that gives up sets the device flag; mra_sync reports MRA_ETIMEOUT.

    The first wait of every consumer warp is shortened to zero polls (the
    copies are real and complete; the kernel waits for them with the normal
    bound before leaving), so no wait can hang.  Rings 1..35 (M = 256) take
    the chunked-staging tensor-core kernel of the split path.
    """
    refs, imgs = _inputs(L, 3, 4, 1.0, 1, seed=31)
    precision = mra.MRA_FP32 if prec == "fp32" else mra.MRA_BF16_RESCORE
    al = mra.Aligner(L, 1, r2, 1, 1.0, 1.0, 1, precision, kernel=kernel)
    al.set_refs(refs.to(DEV))
    good = al.align(imgs.to(DEV))
    mra.mra_sync(al.h)
    os.environ["MRA_DEBUG_FIRST_WAIT_LIMIT"] = "0"
    try:
        al.align(imgs.to(DEV))
        with pytest.raises(mra.MRAError) as ei:
            mra.mra_sync(al.h)
        assert ei.value.code == mra.MRA_ETIMEOUT
    finally:
        del os.environ["MRA_DEBUG_FIRST_WAIT_LIMIT"]
    again = al.align(imgs.to(DEV))
    mra.mra_sync(al.h)
    assert torch.equal(good, again)
    al.close()
