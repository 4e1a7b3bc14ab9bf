"""Pins for the FP64 oracle: checks against mathematics, not against itself.

Each test fixes the oracle to something independent of its own code: a
closed form, a library routine in a special case, a time-domain
re-derivation of the Sec. 2 integral, or exact recovery of a pose built by a
pixel permutation.  A dropped term, a wrong sign or index, a transposed
image axis or a wrong rotation sense fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import mra_oracle as O

RNG = np.random.default_rng(12345)


# ----------------------------------------------------------------------------
# Tables
# ----------------------------------------------------------------------------

def test_ring_table_histograms():
    """N_r = smallest power of two >= 2 pi r: ring-length histogram for rings 1..35 and 1..60."""
    rings = O.ring_table(1, 35, 1)
    hist = {}
    for _, n in rings:
        hist[n] = hist.get(n, 0) + 1
    assert hist == {8: 1, 16: 1, 32: 3, 64: 5, 128: 10, 256: 15}
    assert sum(n for _, n in rings) == 5560
    assert sum(n // 2 + 1 for _, n in rings) == 2815
    assert O.angle_count(rings) == 256
    rings60 = O.ring_table(1, 60, 1)
    assert O.angle_count(rings60) == 512
    assert sum(n for _, n in rings60) == 17080
    assert sum(n // 2 + 1 for _, n in rings60) == 8600
    # ring_step skips radii
    assert [r for r, _ in O.ring_table(3, 11, 4)] == [3, 7, 11]
    with pytest.raises(ValueError):
        O.ring_table(0, 5, 1)


def test_shift_grid_is_sy_major():
    s = O.shift_list(2.0, 1.0)
    assert len(s) == 25
    assert s[0] == (-2.0, -2.0) and s[1] == (-1.0, -2.0) and s[5] == (-2.0, -1.0)
    assert s[12] == (0.0, 0.0)
    assert len(O.shift_list(4.0, 1.0)) == 81 and len(O.shift_list(6.0, 1.0)) == 169
    assert len(O.shift_list(1.0, 0.5)) == 25


# ----------------------------------------------------------------------------
# Library special cases
# ----------------------------------------------------------------------------

def test_bilinear_matches_scipy_grid_constant():
    """Zero-padded bilinear equals scipy's order-1 map_coordinates with grid-constant padding."""
    img = RNG.standard_normal((13, 11))
    x = RNG.uniform(-2.0, 13.0, size=500)
    y = RNG.uniform(-2.0, 15.0, size=500)
    ours = O.bilinear(img, x, y)
    ref = ndi.map_coordinates(img, [y, x], order=1, mode="grid-constant", cval=0.0)
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12)


def test_bilinear_hand_values():
    img = np.array([[1.0, 2.0], [3.0, 5.0]])
    assert O.bilinear(img, np.array([0.5]), np.array([0.5]))[0] == pytest.approx(2.75)
    # x = 1.5 lies between column 1 and the zero column 2
    assert O.bilinear(img, np.array([1.5]), np.array([0.0]))[0] == pytest.approx(1.0)
    assert O.bilinear(img, np.array([-0.25]), np.array([1.0]))[0] == pytest.approx(0.75 * 3.0)


@pytest.mark.parametrize("n", [8, 16, 64, 256])
def test_ring_dft_matches_numpy_fft(n):
    x = RNG.standard_normal(n)
    X = O.ring_dft(x)
    F = np.fft.fft(x)
    for f in range(-n // 2, n // 2 + 1):
        assert abs(X[f + n // 2] - F[f % n]) < 1e-9 * (1 + abs(F[f % n]))


def test_aligned_image_matches_scipy_affine():
    """a(c0+w) = I(c0 + s + Mm R(-phi) w) equals scipy's order-1 affine_transform (zero padding)."""
    L = 24
    img = RNG.standard_normal((L, L))
    c = L / 2.0
    for sx, sy, m, phi in [(1.0, -2.0, 0, 0.7), (-1.5, 0.5, 1, 2.9), (0.0, 0.0, 1, 0.0)]:
        ours = O.aligned_image(img, sx, sy, m, phi)
        cs, sn = math.cos(phi), math.sin(phi)
        # output (row=y, col=x) index -> input index; w = (x - c, y - c)
        # x_in = c + sx + sgn*(cs*wx + sn*wy); y_in = c + sy + (-sn*wx + cs*wy)
        sg = -1.0 if m else 1.0
        A = np.array([[cs, -sn], [sg * sn, sg * cs]])          # rows: (y_in, x_in); cols: (wy, wx)
        off = np.array([c + sy, c + sx]) - A @ np.array([c, c])
        ref = ndi.affine_transform(img, A, offset=off, order=1, mode="grid-constant", cval=0.0)
        np.testing.assert_allclose(ours, ref, atol=1e-10)


# ----------------------------------------------------------------------------
# Closed forms of the Sec. 2 CC on ring arrays
# ----------------------------------------------------------------------------

def _theta(n):
    return 2.0 * math.pi * np.arange(n) / n


@pytest.mark.parametrize("dr", [1, 2])
def test_tone_closed_form(dr):
    """x = cos(a theta), y = cos(a theta + b) on ring r:  c(phi) = pi r dr cos(a phi + b)."""
    rings = [(3, 32), (9, 64)]
    a, b = 5, 0.7
    xs = [np.cos(a * _theta(n)) for _, n in rings]
    ys = [np.cos(a * _theta(n) + b) for _, n in rings]
    c = O.cc_rings(xs, ys, rings, dr)
    phi = 2.0 * math.pi * np.arange(64) / 64
    expect = sum(math.pi * r * dr for r, _ in rings) * np.cos(a * phi + b)
    np.testing.assert_allclose(c, expect, atol=1e-9)


def test_sine_tone_closed_form():
    """x = sin(a theta), y = sin(a theta + b): c(phi) = pi r dr cos(a phi + b)."""
    rings = [(7, 64)]
    a, b = 11, -1.3
    c = O.cc_rings([np.sin(a * _theta(64))], [np.sin(a * _theta(64) + b)], rings, 1)
    phi = 2.0 * math.pi * np.arange(64) / 64
    np.testing.assert_allclose(c, math.pi * 7 * np.cos(a * phi + b), atol=1e-9)


def test_nyquist_tone_on_inner_ring():
    """a = N_r/2 on an inner ring (N_r < M): c = 2 pi r dr cos(b) cos(N_r phi / 2) (pins the 1/2 split)."""
    rings = [(1, 8), (5, 32)]
    b = 0.4
    xs = [np.cos(4 * _theta(8)), np.zeros(32)]
    ys = [np.cos(4 * _theta(8) + b), np.zeros(32)]
    c = O.cc_rings(xs, ys, rings, 1)
    phi = 2.0 * math.pi * np.arange(32) / 32
    np.testing.assert_allclose(c, 2.0 * math.pi * math.cos(b) * np.cos(4 * phi), atol=1e-9)


def test_nyquist_tone_on_outer_ring():
    rings = [(5, 32)]
    b = 1.1
    c = O.cc_rings([np.cos(16 * _theta(32))], [np.cos(16 * _theta(32) + b)], rings, 3)
    phi = 2.0 * math.pi * np.arange(32) / 32
    np.testing.assert_allclose(c, 2.0 * math.pi * 5 * 3 * math.cos(b) * np.cos(16 * phi), atol=1e-9)


def test_dc_closed_form():
    rings = O.ring_table(2, 9, 1)
    xs = [np.ones(n) for _, n in rings]
    c = O.cc_rings(xs, xs, rings, 1)
    np.testing.assert_allclose(c, 2.0 * math.pi * sum(r for r, _ in rings), rtol=1e-12)


# ----------------------------------------------------------------------------
# Time-domain re-derivation (periodic sinc interpolant, Trefethen ch. 3)
# ----------------------------------------------------------------------------

def _periodic_sinc(n, t):
    """S_N(t) = sin(N t / 2) cot(t / 2) / N for even N, S_N(0) = 1."""
    t = np.asarray(t, dtype=np.float64)
    out = np.ones_like(t)
    s = np.sin(t / 2.0)
    nz = np.abs(s) > 1e-14
    out[nz] = np.sin(n * t[nz] / 2.0) * np.cos(t[nz] / 2.0) / (n * s[nz])
    return out


def test_cc_equals_direct_sum_with_sinc_interpolant():
    """c(phi_j) = sum_r dr r (2 pi/N_r) sum_q x_q ytilde_r(theta_q + phi_j), ytilde = periodic-sinc interpolant."""
    rings = O.ring_table(1, 12, 1)          # N_r in 8..128, M = 128
    M = O.angle_count(rings)
    xs = [RNG.standard_normal(n) for _, n in rings]
    ys = [RNG.standard_normal(n) for _, n in rings]
    c = O.cc_rings(xs, ys, rings, 1)
    direct = np.zeros(M)
    for j in range(M):
        phi = 2.0 * math.pi * j / M
        for (r, n), x, y in zip(rings, xs, ys):
            th = _theta(n)
            yt = np.array([np.dot(y, _periodic_sinc(n, tq + phi - th)) for tq in th])
            direct[j] += r * (2.0 * math.pi / n) * np.dot(x, yt)
    np.testing.assert_allclose(c, direct, atol=1e-9 * np.abs(direct).max())


def test_cc_equals_circular_correlation_on_grid_lags():
    """For lags on each ring's own grid the CC is the plain circular correlation."""
    rings = [(21, 256), (30, 256), (35, 256)]
    xs = [RNG.standard_normal(256) for _ in rings]
    ys = [RNG.standard_normal(256) for _ in rings]
    c = O.cc_rings(xs, ys, rings, 1)
    for j in [0, 1, 17, 128, 255]:
        d = sum(r * (2 * math.pi / 256) * np.dot(x, np.roll(y, -j)) for (r, _), x, y in zip(rings, xs, ys))
        assert abs(c[j] - d) < 1e-9 * abs(d) + 1e-9


# ----------------------------------------------------------------------------
# Mirror identity and the self-CC invariant
# ----------------------------------------------------------------------------

def test_mirror_identity_against_direct_resampling():
    """X^(1)(f) = (-1)^f conj(X^(0)(f)) for samples taken at mirrored points."""
    L = 32
    img = RNG.standard_normal((L, L))
    cfg = O.MRAConfig(L, 1, 10, 1, 1.0, 1.0, 1)
    spec = O.particle_spectra(img, cfg)
    for (r, n), X in zip(O.ring_table(1, 10, 1), spec):
        f = np.arange(-n // 2, n // 2 + 1)
        np.testing.assert_allclose(X[:, 1, :], ((-1.0) ** f) * np.conj(X[:, 0, :]), atol=1e-9)


def test_self_cc_peaks_at_zero_angle():
    """An image against itself (s = 0, m = 0) peaks at j = 0 (Cauchy-Schwarz over angles)."""
    L = 40
    rings = O.ring_table(2, 15, 1)
    for _ in range(3):
        img = RNG.standard_normal((L, L))
        xs = O.polar_samples(img, rings)
        c = O.cc_rings(xs, xs, rings, 1)
        assert int(np.argmax(c)) == 0
        assert c[0] == pytest.approx(sum(r * 2 * math.pi / n * np.dot(x, x)
                                         for (r, n), x in zip(rings, xs)), rel=1e-12)


def test_tie_break_smallest_index():
    cfg = O.MRAConfig(16, 1, 2, 1, 1.0, 1.0, 1)
    c = np.zeros((2, 9, 2, 16))
    c[1, 3, 0, 5] = 2.0
    c[0, 7, 1, 2] = 2.0
    c[0, 7, 1, 9] = 2.0
    p = O._pose_from_table(c, cfg)
    assert (p.k, p.shift_idx, p.mirror, p.ang_idx) == (0, 7, 1, 2)
    assert p.runner_up == 2.0


# ----------------------------------------------------------------------------
# Exact pose recovery from pixel permutations (quarter turns, integer shifts, mirror)
# ----------------------------------------------------------------------------

def _compact_refs(K, L, seed):
    """Blob references vanishing outside a disc of radius 9 about c0 (so permutations stay exact)."""
    rng = np.random.default_rng(seed)
    c = L / 2.0
    yy, xx = np.meshgrid(np.arange(L) - c, np.arange(L) - c, indexing="ij")
    refs = np.zeros((K, L, L))
    for k in range(K):
        for _ in range(6):
            cx, cy = rng.uniform(-5, 5, size=2)
            s = rng.uniform(1.2, 2.5)
            refs[k] += rng.uniform(0.5, 1.5) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
        refs[k][xx ** 2 + yy ** 2 > 81] = 0.0
    return refs


def _permute(ref, quarter, tx, ty, m):
    """I(c0 + u) = ref(c0 + R(-alpha)(Mm u - t)), alpha = quarter * 90 deg, on integer offsets."""
    L = ref.shape[0]
    c = L // 2
    out = np.zeros_like(ref)
    ca = [1, 0, -1, 0][quarter % 4]
    sa = [0, 1, 0, -1][quarter % 4]
    for y in range(L):
        for x in range(L):
            ux, uy = x - c, y - c
            if m:
                ux = -ux
            vx, vy = ux - tx, uy - ty
            px = ca * vx + sa * vy          # R(-alpha) v
            py = -sa * vx + ca * vy
            X, Y = px + c, py + c
            if 0 <= X < L and 0 <= Y < L:
                out[y, x] = ref[Y, X]
    return out


@pytest.mark.parametrize("quarter,tx,ty,m", [(1, 2, -1, 0), (3, -1, 2, 1), (2, 0, 1, 1), (0, 1, 1, 0)])
def test_exact_recovery_of_permuted_reference(quarter, tx, ty, m):
    L = 32
    refs = _compact_refs(3, L, seed=7)
    k = 1
    cfg = O.MRAConfig(L, 1, 8, 1, 2.0, 1.0, 1)
    img = _permute(refs[k], quarter, tx, ty, m)
    ref_spec = O.reference_spectra(refs, cfg)
    c = O.cc_table(img, ref_spec, cfg)
    p = O._pose_from_table(c, cfg)
    M = c.shape[-1]
    ex_sx = -tx if m else tx                      # s = Mm t
    assert (p.k, p.mirror) == (k, m)
    assert (p.sx, p.sy) == (float(ex_sx), float(ty))
    assert p.ang_idx == (-quarter * M // 4) % M
    rings = O.ring_table(1, 8, 1)
    xs = O.polar_samples(refs[k], rings)
    self_cc = O.cc_rings(xs, xs, rings, 1)[0]
    assert p.cc == pytest.approx(self_cc, rel=1e-10)
    # Averaging pin: the aligned particle is the reference itself on the grid.
    a = O.aligned_image(img, p.sx, p.sy, p.mirror, 2 * math.pi * p.ang_idx / M)
    np.testing.assert_allclose(a, refs[k], atol=1e-9)
    avg, cnt = O.average(np.stack([img, img]), [p, p], 3, M)
    assert list(cnt) == [0, 2, 0]
    np.testing.assert_allclose(avg[1], refs[k], atol=1e-9)
    assert np.isnan(avg[0]).all()


# ----------------------------------------------------------------------------
# Analytic recovery and the brute-force CC (pins rotation sense and shift sign)
# ----------------------------------------------------------------------------

def _blob_fn(cx, cy, s, a, L):
    c = L / 2.0

    def f(x, y):
        x = np.asarray(x) - c
        y = np.asarray(y) - c
        return sum(ai * np.exp(-((x - xi) ** 2 + (y - yi) ** 2) / (2 * si * si))
                   for xi, yi, si, ai in zip(cx, cy, s, a))
    return f


def test_analytic_recovery_and_bruteforce():
    L = 48
    rng = np.random.default_rng(99)
    K = 2
    params = []
    refs = np.zeros((K, L, L))
    ys, xs = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    for k in range(K):
        cx, cy = rng.uniform(-8, 8, size=(2, 8))
        s = rng.uniform(2.5, 4.0, size=8)
        a = rng.uniform(0.5, 1.5, size=8)
        raw = _blob_fn(cx, cy, s, a, L)(xs, ys)
        params.append((cx, cy, s, a, raw.mean(), raw.std()))
        refs[k] = (raw - raw.mean()) / raw.std()
    cfg = O.MRAConfig(L, 2, 16, 1, 2.0, 1.0, 1)
    M = O.angle_count(O.ring_table(2, 16, 1))
    ref_spec = O.reference_spectra(refs, cfg)
    for (k, j0, tx, ty, m) in [(0, 37, 1, -2, 0), (1, 5, -2, 1, 1), (1, 100, 0, 2, 1)]:
        alpha = 2 * math.pi * j0 / M
        cx, cy, s, a, mu, sd = params[k]
        # particle blob centres: Mm (t + R(alpha) c)
        ex = math.cos(alpha) * cx - math.sin(alpha) * cy + tx
        ey = math.sin(alpha) * cx + math.cos(alpha) * cy + ty
        if m:
            ex = -ex
        img = (_blob_fn(ex, ey, s, a, L)(xs, ys) - mu) / sd
        # Raw CC does not rank classes by a theorem (another blob cluster may
        # correlate more over the annulus), so the pose is checked within the
        # true class; class choice is pinned by the permutation test above.
        c = O.cc_table(img, ref_spec, cfg)[k:k + 1]
        p = O._pose_from_table(c, cfg)
        assert (p.mirror, p.ang_idx) == (m, (-j0) % M)
        assert (p.sx, p.sy) == (float(-tx if m else tx), float(ty))
        blob = _blob_fn(cx, cy, s, a, L)
        bf = O.cc_bruteforce(img, lambda x, y: (blob(x, y) - mu) / sd, cfg, p.sx, p.sy, p.mirror)
        row = c[0, p.shift_idx, p.mirror]
        assert int(np.argmax(bf)) == p.ang_idx
        assert np.max(np.abs(row - bf)) <= 1e-2 * np.max(np.abs(bf))


# ----------------------------------------------------------------------------
# Reference spectra from the table path agree with the ring-array path
# ----------------------------------------------------------------------------

def test_cc_table_consistent_with_cc_rings():
    L = 28
    img = RNG.standard_normal((L, L))
    refs = RNG.standard_normal((2, L, L))
    cfg = O.MRAConfig(L, 1, 9, 2, 1.0, 1.0, 1)
    rings = O.ring_table(1, 9, 2)
    c = O.cc_table(img, O.reference_spectra(refs, cfg), cfg)
    for k in range(2):
        yk = O.polar_samples(refs[k], rings)
        for si, (sx, sy) in enumerate(O.shift_list(1.0, 1.0)):
            for m in (0, 1):
                xk = O.polar_samples(img, rings, sx, sy, m)
                np.testing.assert_allclose(c[k, si, m], O.cc_rings(xk, yk, rings, 2), atol=1e-9)


# ----------------------------------------------------------------------------
# Classification loop: normalisation and the fixed point of one pass
# ----------------------------------------------------------------------------

def test_normalize_invariants():
    x = RNG.standard_normal((20, 20)) * 3.0 + 2.0
    z = O.normalize(x)
    assert abs(z.mean()) < 1e-12
    assert math.sqrt(np.mean(z * z)) == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(O.normalize(5.0 * x - 7.0), z, atol=1e-12)   # affine invariance (a > 0)
    np.testing.assert_allclose(O.normalize(-x), -z, atol=1e-12)             # odd under negation
    assert np.array_equal(O.normalize(np.full((6, 6), 4.5)), np.zeros((6, 6)))
    # library routine in a special case: population standard deviation
    np.testing.assert_allclose(z, (x - x.mean()) / np.std(x, ddof=0), atol=1e-12)


def test_refresh_rules():
    refs = RNG.standard_normal((3, 8, 8))
    avg = RNG.standard_normal((3, 8, 8)) + 1.0
    imgs = RNG.standard_normal((4, 8, 8))
    out = O.refresh_refs(refs, avg, np.array([2, 0, 0]), np.array([-1, 3, -1]), imgs)
    np.testing.assert_allclose(out[0], O.normalize(avg[0]))
    np.testing.assert_allclose(out[1], O.normalize(imgs[3]))
    assert np.array_equal(out[2], refs[2])


def test_classification_pass_fixed_point():
    """Particles that are exact grid permutations of compact references: one
    pass assigns every particle to its source class and returns the
    normalised references (the aligned particles are the references pixel for
    pixel, so every class average is its reference).  The references are
    scaled to equal ring-weighted energy E: by Cauchy-Schwarz on the ring
    spectra (Parseval with the split Nyquist term) any other class scores at
    most E, which the source class reaches exactly."""
    L = 32
    refs = _compact_refs(3, L, seed=17)
    rings = O.ring_table(1, 8, 1)
    for k in range(3):
        xs = O.polar_samples(refs[k], rings)
        refs[k] /= math.sqrt(O.cc_rings(xs, xs, rings, 1)[0])
    cfg = O.MRAConfig(L, 1, 8, 1, 1.0, 1.0, 1)
    cases = [(0, 1, 1, 0, 0), (1, 3, 0, -1, 1), (2, 2, -1, 1, 1), (1, 0, 1, 0, 0), (2, 1, 0, 0, 0)]
    imgs = np.stack([_permute(refs[k], q, tx, ty, m) for k, q, tx, ty, m in cases])
    poses, new_refs, counts = O.classify_iteration(imgs, refs, cfg)
    assert [p.k for p in poses] == [c[0] for c in cases]
    assert list(counts) == [1, 2, 2]
    want = (refs - refs.mean(axis=(1, 2), keepdims=True)) / refs.std(axis=(1, 2), keepdims=True)
    np.testing.assert_allclose(new_refs, want, atol=1e-9)
