"""FP64 CPU oracle for polar-resampling multi-reference alignment (MRA).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant with the CUDA library: it has its own ring table,
its own bilinear interpolation, explicit DFT sums (no FFT) and its own angle
grid, all in float64.

What it computes (Cryo-RALib, arXiv 2011.05755):

* Sec. 2 defines the rotational cross-correlation of a particle x and a
  reference y in polar coordinates,
  ``c(phi) = int_{r1}^{r2} int_0^{2 pi} x(r, theta) y(r, theta + phi) |r| dtheta dr``,
  and Algorithm 1 (Sec. 3) evaluates it for every reference, every shift on
  the search grid and both mirror states, then takes the table maximum per
  image (Fig. 2 / Sec. 3 reduction) and rebuilds the class averages from the
  aligned images.
* Quadrature (reading, as the paper gives only the integral): rings
  ``r = r1, r1 + dr, ..., r2`` with ``N_r`` = the smallest power of two
  ``>= 2 pi r`` samples at ``theta_q = 2 pi q / N_r``; a Riemann sum with weight
  ``dr * r * 2 pi / N_r`` per sample; the reference ring is continued between
  its samples by its trigonometric interpolant with the Nyquist term split
  equally between +-N_r/2.  In the Fourier domain this is
  ``c(phi) = sum_r (2 pi r dr / N_r^2) sum_{f=-N_r/2}^{N_r/2} eps_f conj(X_r(f)) Y_r(f) e^{i f phi}``
  with ``eps_{+-N_r/2} = 1/2``, ``X(f) = sum_q x_q e^{-2 pi i f q / N_r}``; it is
  evaluated at ``phi_j = 2 pi j / M``, ``M = max_r N_r``.
* Geometry (reading): box centre ``c0 = (L/2, L/2)``; image ``[y][x]``;
  bilinear interpolation with every neighbour outside ``[0, L-1]^2`` read as
  zero; particle samples at ``c0 + s + Mm r (cos theta, sin theta)`` with the
  mirror ``Mm = diag(-1, 1)^m`` applied to the ring offset after the shift.
* Pose: argmax over ``(k, s, m, j)``; among bit-equal values the smallest
  ``(k, shift index, m, j)`` in lexicographic order wins.  The aligned image
  is ``a(c0 + w) = I(c0 + s + Mm R(-phi) w)``.

Every function is written from those definitions; none is tuned for speed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

__all__ = [
    "MRAConfig", "Pose", "ring_table", "angle_count", "shift_list", "bilinear",
    "ring_offsets", "polar_samples", "ring_dft", "ring_weights", "cc_rings",
    "cc_table", "reference_spectra", "particle_spectra", "align", "align_one",
    "aligned_image", "average", "normalize", "refresh_refs", "classify_iteration",
    "cc_bruteforce",
]


@dataclasses.dataclass(frozen=True)
class MRAConfig:
    """Search configuration (rings, shift grid, mirror) for a box of size L."""
    L: int
    first_ring: int
    last_ring: int
    ring_step: int = 1
    shift_range: float = 0.0
    shift_step: float = 1.0
    mirror: int = 1


@dataclasses.dataclass
class Pose:
    """Best pose of one particle, and its CC gap to the runner-up."""
    k: int
    shift_idx: int
    mirror: int
    ang_idx: int
    sx: float
    sy: float
    angle_deg: float
    cc: float
    runner_up: float

    @property
    def rel_gap(self) -> float:
        return (self.cc - self.runner_up) / abs(self.cc) if self.cc != 0 else 0.0


# ---------------------------------------------------------------------------
# Tables (Sec. 2 integral -> sampled rings; reading of the quadrature)
# ---------------------------------------------------------------------------

def ring_table(first_ring: int, last_ring: int, ring_step: int = 1) -> List[tuple]:
    """Rings ``(r, N_r)``: r = r1, r1+dr, ..., r2 and N_r the smallest power of two >= 2 pi r."""
    if first_ring < 1 or last_ring < first_ring or ring_step < 1:
        raise ValueError("rings need 1 <= first_ring <= last_ring and ring_step >= 1")
    out = []
    for r in range(first_ring, last_ring + 1, ring_step):
        n = 1
        while n < 2.0 * math.pi * r:
            n *= 2
        out.append((r, n))
    return out


def angle_count(rings: Sequence[tuple]) -> int:
    """M: number of in-plane angles searched, the largest ring length."""
    return max(n for _, n in rings)


def shift_list(shift_range: float, shift_step: float) -> List[tuple]:
    """Shift grid ``(sx, sy)``, each axis -R, -R+d, ..., R; index = iy * nx + ix (sy-major)."""
    cnt = int(round(2.0 * shift_range / shift_step)) + 1
    axis = [-shift_range + i * shift_step for i in range(cnt)]
    return [(sx, sy) for sy in axis for sx in axis]


def ring_weights(rings: Sequence[tuple], ring_step: int) -> np.ndarray:
    """Quadrature weight per sample on ring r: dr * r * (2 pi / N_r)."""
    return np.array([ring_step * r * 2.0 * math.pi / n for r, n in rings])


# ---------------------------------------------------------------------------
# Polar conversion (Alg. 1, shift-loop conversion step: resampling on the rings
# about the shifted centre)
# ---------------------------------------------------------------------------

def bilinear(img: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of ``img[y][x]`` at real points, zero outside the box.

    x0 = floor(x), fx = x - x0 (same for y); each of the four neighbours that
    falls outside [0, L-1]^2 contributes zero.
    """
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    x0 = np.floor(x)
    y0 = np.floor(y)
    fx = x - x0
    fy = y - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    out = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    for dx, dy, w in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)),
                      (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
        xi = x0 + dx
        yi = y0 + dy
        inside = (xi >= 0) & (xi < W) & (yi >= 0) & (yi < H)
        vals = np.where(inside, img[np.clip(yi, 0, H - 1), np.clip(xi, 0, W - 1)], 0.0)
        out += w * vals
    return out


def ring_offsets(r: int, n: int):
    """Unit-ring sample offsets ``r (cos theta_q, sin theta_q)``, theta_q = 2 pi q / n."""
    theta = 2.0 * math.pi * np.arange(n) / n
    return r * np.cos(theta), r * np.sin(theta)


def polar_samples(img: np.ndarray, rings: Sequence[tuple], sx: float = 0.0, sy: float = 0.0,
                  mirror: int = 0) -> List[np.ndarray]:
    """Samples ``x_r(theta_q) = I(c0 + s + Mm r (cos theta_q, sin theta_q))`` for every ring."""
    L = img.shape[0]
    c = L / 2.0
    out = []
    for r, n in rings:
        ox, oy = ring_offsets(r, n)
        if mirror:
            ox = -ox
        out.append(bilinear(img, c + sx + ox, c + sy + oy))
    return out


# ---------------------------------------------------------------------------
# Ring spectra and the CC (Sec. 2 definition, sampled)
# ---------------------------------------------------------------------------

def ring_dft(x: np.ndarray) -> np.ndarray:
    """Explicit DFT ``X(f) = sum_q x_q exp(-2 pi i f q / N)`` for f = -N/2 .. N/2.

    Works on the last axis; returns N+1 bins, index f + N/2.
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[-1]
    f = np.arange(-n // 2, n // 2 + 1)
    q = np.arange(n)
    F = np.exp(-2j * math.pi * np.outer(f, q) / n)      # [N+1, N]
    return x @ F.T


def _eps(n: int) -> np.ndarray:
    """Nyquist split of the trigonometric interpolant: 1/2 at f = +-N/2, 1 elsewhere."""
    e = np.ones(n + 1)
    e[0] = e[-1] = 0.5
    return e


def cc_rings(x_rings: Sequence[np.ndarray], y_rings: Sequence[np.ndarray],
             rings: Sequence[tuple], ring_step: int, M: Optional[int] = None) -> np.ndarray:
    """CC ``c(phi_j)``, j = 0..M-1, between two sets of ring samples (spectral form of the Sec. 2 integral).

    ``x_rings`` / ``y_rings``: one array of N_r samples per ring (leading batch
    axes allowed and broadcast against each other).
    """
    M = angle_count(rings) if M is None else M
    C = None
    for (r, n), xr, yr in zip(rings, x_rings, y_rings):
        X = ring_dft(xr)
        Y = ring_dft(yr)
        term = (2.0 * math.pi * r * ring_step / n ** 2) * _eps(n) * np.conj(X) * Y
        if C is None:
            C = np.zeros(term.shape[:-1] + (M + 1,), dtype=np.complex128)
        C[..., M // 2 - n // 2: M // 2 + n // 2 + 1] += term
    f = np.arange(-M // 2, M // 2 + 1)
    phi = 2.0 * math.pi * np.arange(M) / M
    E = np.exp(1j * np.outer(f, phi))                     # [M+1, M]
    c = C @ E
    return c.real


def reference_spectra(refs: np.ndarray, cfg: MRAConfig) -> List[np.ndarray]:
    """Per ring, the DFT of every reference's unshifted polar samples: list of [K, N_r+1]."""
    rings = ring_table(cfg.first_ring, cfg.last_ring, cfg.ring_step)
    per_ref = [polar_samples(ref, rings) for ref in refs]
    return [ring_dft(np.stack([pr[i] for pr in per_ref])) for i in range(len(rings))]


def particle_spectra(img: np.ndarray, cfg: MRAConfig) -> List[np.ndarray]:
    """Per ring, the DFT of the particle's samples at every shift and mirror: list of [S, 2, N_r+1].

    Mirrored samples are resampled directly at the reflected points.
    """
    rings = ring_table(cfg.first_ring, cfg.last_ring, cfg.ring_step)
    mirrors = (0, 1) if cfg.mirror else (0,)
    samp = [[polar_samples(img, rings, sx, sy, m) for m in mirrors]
            for sx, sy in shift_list(cfg.shift_range, cfg.shift_step)]
    out = []
    for i in range(len(rings)):
        x = np.stack([np.stack([samp[s][m][i] for m in range(len(mirrors))])
                      for s in range(len(samp))])
        out.append(ring_dft(x))
    return out


def cc_table(img: np.ndarray, ref_spec: List[np.ndarray], cfg: MRAConfig) -> np.ndarray:
    """The paper's CC table row for one image: ``c[k, s, m, j]`` (Sec. 2 table, Algorithm 1)."""
    rings = ring_table(cfg.first_ring, cfg.last_ring, cfg.ring_step)
    M = angle_count(rings)
    xs = particle_spectra(img, cfg)
    C = None
    for (r, n), X, Y in zip(rings, xs, ref_spec):
        wt = (2.0 * math.pi * r * cfg.ring_step / n ** 2) * _eps(n)
        term = np.conj(X)[None, :, :, :] * (Y * wt)[:, None, None, :]   # [K, S, m, N+1]
        if C is None:
            C = np.zeros(term.shape[:-1] + (M + 1,), dtype=np.complex128)
        C[..., M // 2 - n // 2: M // 2 + n // 2 + 1] += term
    f = np.arange(-M // 2, M // 2 + 1)
    phi = 2.0 * math.pi * np.arange(M) / M
    E = np.exp(1j * np.outer(f, phi))
    return C.real @ E.real - C.imag @ E.imag


# ---------------------------------------------------------------------------
# Max reduction and parameters (Algorithm 1 reduction; Fig. 2)
# ---------------------------------------------------------------------------

def _pose_from_table(c: np.ndarray, cfg: MRAConfig) -> Pose:
    M = c.shape[-1]
    flat = c.reshape(-1)
    i = int(np.argmax(flat))                  # first maximum = smallest (k, s, m, j)
    k, s, m, j = np.unravel_index(i, c.shape)
    runner = np.partition(flat, -2)[-2] if flat.size > 1 else -np.inf
    sx, sy = shift_list(cfg.shift_range, cfg.shift_step)[s]
    return Pose(int(k), int(s), int(m), int(j), float(sx), float(sy), 360.0 * j / M,
                float(flat[i]), float(runner))


def align_one(img: np.ndarray, ref_spec: List[np.ndarray], cfg: MRAConfig) -> Pose:
    """Best (reference, shift, mirror, angle) of one particle."""
    return _pose_from_table(cc_table(img, ref_spec, cfg), cfg)


def align(imgs: np.ndarray, refs: np.ndarray, cfg: MRAConfig) -> List[Pose]:
    """Algorithm 1, one pass: poses of every particle against every reference."""
    ref_spec = reference_spectra(np.asarray(refs, dtype=np.float64), cfg)
    return [align_one(np.asarray(im, dtype=np.float64), ref_spec, cfg) for im in imgs]


# ---------------------------------------------------------------------------
# Class averages (Algorithm 1: apply parameters, compute new averages)
# ---------------------------------------------------------------------------

def aligned_image(img: np.ndarray, sx: float, sy: float, mirror: int, angle_rad: float) -> np.ndarray:
    """``a(c0 + w) = I(c0 + s + Mm R(-phi) w)`` on the integer grid w, bilinear, zero outside."""
    L = img.shape[0]
    c = L / 2.0
    wy, wx = np.meshgrid(np.arange(L) - c, np.arange(L) - c, indexing="ij")
    cs, sn = math.cos(angle_rad), math.sin(angle_rad)
    rx = cs * wx + sn * wy
    ry = -sn * wx + cs * wy
    if mirror:
        rx = -rx
    return bilinear(img, c + sx + rx, c + sy + ry)


def average(imgs: np.ndarray, poses: Sequence, K: int, M: int):
    """Class averages ``avg_k = mean of aligned images with class k``; returns ``(avg, counts)``.

    ``poses`` items need ``k, sx, sy, mirror, ang_idx``.  An empty class has
    count 0 and an all-NaN average (the library leaves it untouched).
    """
    L = imgs.shape[-1]
    sums = np.zeros((K, L, L))
    counts = np.zeros(K, dtype=np.int64)
    for img, p in zip(imgs, poses):
        a = aligned_image(np.asarray(img, dtype=np.float64), p.sx, p.sy, p.mirror,
                          2.0 * math.pi * p.ang_idx / M)
        sums[p.k] += a
        counts[p.k] += 1
    avg = np.full((K, L, L), np.nan)
    nz = counts > 0
    avg[nz] = sums[nz] / counts[nz, None, None]
    return avg, counts


def normalize(img: np.ndarray) -> np.ndarray:
    """Zero mean, unit standard deviation over the box (``1/L^2`` variance).

    Reading: the classification loop of Algorithm 1 feeds the class averages
    back as references; their scale is not fixed by the paper, so every new
    reference is brought to mean 0 and standard deviation 1 (a constant image
    becomes all zero) so that the cross-correlation maximum compares classes
    on an equal footing.
    """
    x = np.asarray(img, dtype=np.float64)
    d = x - x.mean()
    var = float(np.mean(d * d))
    return d / math.sqrt(var) if var > 0.0 else np.zeros_like(d)


def refresh_refs(refs: np.ndarray, avg: np.ndarray, counts: np.ndarray, reseed: Optional[np.ndarray] = None,
                 imgs: Optional[np.ndarray] = None) -> np.ndarray:
    """Next references of the classification loop (outer loop of Algorithm 1).

    Class k with ``counts[k] > 0`` becomes ``normalize(avg[k])``; an empty class
    with ``reseed[k] >= 0`` becomes ``normalize(imgs[reseed[k]])``; any other
    class keeps ``refs[k]`` unchanged.
    """
    out = np.array(refs, dtype=np.float64, copy=True)
    for k in range(out.shape[0]):
        if counts[k] > 0:
            out[k] = normalize(avg[k])
        elif reseed is not None and reseed[k] >= 0:
            out[k] = normalize(imgs[reseed[k]])
    return out


def classify_iteration(imgs: np.ndarray, refs: np.ndarray, cfg: MRAConfig, reseed: Optional[np.ndarray] = None):
    """One pass of the classification loop: align, average, refresh.

    Returns ``(poses, new_refs, counts)``.
    """
    poses = align(imgs, refs, cfg)
    M = angle_count(ring_table(cfg.first_ring, cfg.last_ring, cfg.ring_step))
    avg, counts = average(imgs, poses, refs.shape[0], M)
    return poses, refresh_refs(refs, avg, counts, reseed, imgs), counts


# ---------------------------------------------------------------------------
# Brute force (independent of the spectral form): direct sum against a
# reference evaluated exactly at the rotated sample points.
# ---------------------------------------------------------------------------

def cc_bruteforce(img: np.ndarray, ref_fn: Callable[[np.ndarray, np.ndarray], np.ndarray],
                  cfg: MRAConfig, sx: float, sy: float, mirror: int) -> np.ndarray:
    """``sum_r dr r (2 pi / N_r) sum_q x_q y(c0 + r e(theta_q + phi_j))`` for every j.

    ``ref_fn(x, y)`` evaluates the reference at arbitrary points (e.g. an
    analytic blob image).  Agrees with the spectral CC up to interpolation error.
    """
    rings = ring_table(cfg.first_ring, cfg.last_ring, cfg.ring_step)
    M = angle_count(rings)
    L = img.shape[0]
    c0 = L / 2.0
    xs = polar_samples(np.asarray(img, dtype=np.float64), rings, sx, sy, mirror)
    out = np.zeros(M)
    for j in range(M):
        phi = 2.0 * math.pi * j / M
        acc = 0.0
        for (r, n), x in zip(rings, xs):
            th = 2.0 * math.pi * np.arange(n) / n + phi
            y = ref_fn(c0 + r * np.cos(th), c0 + r * np.sin(th))
            acc += cfg.ring_step * r * (2.0 * math.pi / n) * float(np.dot(x, y))
        out[j] = acc
    return out
