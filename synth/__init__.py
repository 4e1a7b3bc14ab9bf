"""Seeded synthetic particle stacks for multi-reference alignment (MRA).

This module makes inputs only.  It holds none of the alignment arithmetic
(no polar resampling, no ring transforms, no cross-correlation): both the
FP64 oracle and the CUDA path read the images it writes, so it is the one
piece of code the two sides share.

Model (the paper's workload is a down-sampled 80S ribosome stack, Sec. 5,
which is not available; these blob images stand in for it):

* A reference is a sum of G isotropic Gaussians ``a * exp(-|u - c|^2 / 2 s^2)``
  point-sampled at the integer pixel positions, with ``s ~ U[s_lo, s_hi]``,
  ``a ~ U[a_lo, a_hi]`` and the centre ``c`` uniform in a disc of radius
  ``disc`` about the box centre ``c0 = (L/2, L/2)``.  Each reference is then
  normalised to zero mean and unit standard deviation over the box.
* A particle picks a reference ``k``, an angle ``alpha ~ U[0, 2 pi)``, an
  integer shift ``t`` in ``[-T, T]^2`` and a mirror bit ``m ~ Bernoulli(1/2)``
  and is rendered analytically as ``I(c0 + u) = ref_k(c0 + R(-alpha)(Mm u - t))``
  with ``Mm = diag(-1, 1)^m`` (rotate by alpha, shift by t, then mirror
  x -> -x), by moving the blob centres to ``Mm (t + R(alpha)(c - c0))``.  The
  rendered signal gets its reference's affine normalisation, white Gaussian
  noise of variance ``var_box(signal) / snr`` is added, and the particle is
  normalised to zero mean and unit standard deviation.

Images are row-major ``[y][x]`` with ``x`` the fast axis.  Parameters come
from numpy's PCG64 (seeded); rendering and noise use torch in float64 on the
requested device (the noise stream therefore depends on the device type).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import torch

__all__ = [
    "Workload", "WORKLOADS", "BlobRefs", "ParticleTruth",
    "make_refs", "draw_particle_truth", "render_particles", "make_particles",
    "make_workload", "shift_grid",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic MRA workload: stack size, box, references, search grid."""
    name: str
    n: int
    L: int
    K: int
    blobs: int
    sigma: tuple
    amp: tuple
    disc: float
    snr: float
    first_ring: int
    last_ring: int
    ring_step: int
    shift_range: float
    shift_step: float
    mirror: int
    seed_refs: int
    seed_particles: int
    seed_noise: int


# The three stack workloads of the measurement plan, named by their sizes.
WORKLOADS = {
    w.name: w for w in [
        Workload("mra_n500_L76_K10_shift2", 500, 76, 10, 20, (3.0, 8.0), (0.5, 1.5), 28.0,
                 0.1, 1, 35, 1, 2.0, 1.0, 1, 1001, 2001, 3001),
        Workload("mra_n100k_L76_K100_shift4", 100_000, 76, 100, 20, (3.0, 8.0), (0.5, 1.5),
                 28.0, 0.1, 1, 35, 1, 4.0, 1.0, 1, 1002, 2002, 3002),
        Workload("mra_n50k_L128_K200_shift6", 50_000, 128, 200, 40, (4.0, 12.0), (0.5, 1.5),
                 50.0, 0.05, 1, 60, 1, 6.0, 1.0, 1, 1003, 2003, 3003),
    ]
}


@dataclasses.dataclass
class BlobRefs:
    """Blob parameters of K references plus their box normalisation."""
    L: int
    centres: np.ndarray   # [K, G, 2] offsets from c0, (x, y)
    sigma: np.ndarray     # [K, G]
    amp: np.ndarray       # [K, G]
    mean: np.ndarray      # [K] box mean of the raw rendering
    std: np.ndarray       # [K] box std of the raw rendering


@dataclasses.dataclass
class ParticleTruth:
    """Ground-truth pose of each particle (generator convention)."""
    k: np.ndarray         # [n] reference index
    alpha: np.ndarray     # [n] rotation angle (radians)
    t: np.ndarray         # [n, 2] integer shift (tx, ty)
    m: np.ndarray         # [n] mirror bit


def shift_grid(shift_range: float, shift_step: float):
    """Search-grid offsets along one axis: -R, -R + d, ..., R (count 2R/d + 1)."""
    cnt = int(round(2.0 * shift_range / shift_step)) + 1
    return [-shift_range + i * shift_step for i in range(cnt)]


def _render(centres: torch.Tensor, sigma: torch.Tensor, amp: torch.Tensor, L: int) -> torch.Tensor:
    """Sum of isotropic Gaussians on the integer pixel grid, separably.

    centres [B, G, 2] are offsets from c0 = (L/2, L/2); returns [B, L, L] (y, x).
    """
    grid = torch.arange(L, dtype=torch.float64, device=centres.device) - L / 2.0
    inv = 1.0 / (2.0 * sigma * sigma)                                  # [B, G]
    ex = torch.exp(-(grid[None, None, :] - centres[..., 0:1]) ** 2 * inv[..., None])
    ey = torch.exp(-(grid[None, None, :] - centres[..., 1:2]) ** 2 * inv[..., None])
    return torch.einsum("bg,bgy,bgx->byx", amp, ey, ex)


def make_refs(K: int, L: int, blobs: int = 20, sigma=(3.0, 8.0), amp=(0.5, 1.5),
              disc: float = 28.0, seed: int = 1001, device="cpu"):
    """K blob references, each normalised to zero mean / unit std over the box.

    Returns ``(refs [K, L, L] float64 torch tensor, BlobRefs)``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    s = rng.uniform(sigma[0], sigma[1], size=(K, blobs))
    a = rng.uniform(amp[0], amp[1], size=(K, blobs))
    rho = disc * np.sqrt(rng.uniform(0.0, 1.0, size=(K, blobs)))
    psi = rng.uniform(0.0, 2.0 * math.pi, size=(K, blobs))
    c = np.stack([rho * np.cos(psi), rho * np.sin(psi)], axis=-1)
    raw = _render(torch.tensor(c, device=device), torch.tensor(s, device=device),
                  torch.tensor(a, device=device), L)
    mean = raw.mean(dim=(1, 2))
    std = raw.std(dim=(1, 2), unbiased=False)
    refs = (raw - mean[:, None, None]) / std[:, None, None]
    return refs, BlobRefs(L, c, s, a, mean.cpu().numpy(), std.cpu().numpy())


def draw_particle_truth(n: int, K: int, shift_range: int, mirror: bool, seed: int) -> ParticleTruth:
    """Uniform reference, angle, integer shift in [-T, T]^2 and fair mirror bit."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, K, size=n)
    alpha = rng.uniform(0.0, 2.0 * math.pi, size=n)
    T = int(shift_range)
    t = rng.integers(-T, T + 1, size=(n, 2))
    m = rng.integers(0, 2, size=n) if mirror else np.zeros(n, dtype=np.int64)
    return ParticleTruth(k, alpha, t, m)


def render_particles(refs: BlobRefs, truth: ParticleTruth, *, snr: Optional[float],
                     noise_seed: int = 3001, normalise: bool = True, device="cpu",
                     out: Optional[torch.Tensor] = None, batch: int = 8192) -> torch.Tensor:
    """Render particles analytically from their references' blobs.

    A particle with pose (k, alpha, t, m) has its blob centres at
    ``Mm (t + R(alpha) (c - c0))``.  ``snr=None`` adds no noise.  With
    ``normalise`` the final image has zero mean and unit std over the box.
    Returns float64 ``[n, L, L]`` unless ``out`` (any float dtype/device) is given.
    """
    n, L = len(truth.k), refs.L
    if out is None:
        out = torch.empty((n, L, L), dtype=torch.float64, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(noise_seed)
    for b0 in range(0, n, batch):
        b1 = min(n, b0 + batch)
        k = truth.k[b0:b1]
        ca, sa = np.cos(truth.alpha[b0:b1]), np.sin(truth.alpha[b0:b1])
        d = refs.centres[k]                                            # [B, G, 2]
        rx = ca[:, None] * d[..., 0] - sa[:, None] * d[..., 1] + truth.t[b0:b1, 0:1]
        ry = sa[:, None] * d[..., 0] + ca[:, None] * d[..., 1] + truth.t[b0:b1, 1:2]
        sign = np.where(truth.m[b0:b1] == 1, -1.0, 1.0)
        e = np.stack([sign[:, None] * rx, ry], axis=-1)
        img = _render(torch.tensor(e, device=device), torch.tensor(refs.sigma[k], device=device),
                      torch.tensor(refs.amp[k], device=device), L)
        img = (img - torch.tensor(refs.mean[k], device=device)[:, None, None]) \
            / torch.tensor(refs.std[k], device=device)[:, None, None]
        if snr is not None:
            var = img.var(dim=(1, 2), unbiased=False)
            noise = torch.randn(img.shape, generator=gen, dtype=torch.float64, device=device)
            img = img + noise * torch.sqrt(var / snr)[:, None, None]
        if normalise:
            img = (img - img.mean(dim=(1, 2), keepdim=True)) / img.std(dim=(1, 2), unbiased=False,
                                                                         keepdim=True)
        out[b0:b1].copy_(img)
    return out


def make_particles(refs: BlobRefs, n: int, *, shift_range: int, mirror: bool, snr: Optional[float],
                   seed: int = 2001, noise_seed: int = 3001, device="cpu", out=None):
    """Draw poses and render ``n`` particles; returns ``(images, truth)``."""
    truth = draw_particle_truth(n, len(refs.sigma), shift_range, mirror, seed)
    imgs = render_particles(refs, truth, snr=snr, noise_seed=noise_seed, device=device, out=out)
    return imgs, truth


def make_workload(w: Workload, n: Optional[int] = None, device="cpu", dtype=torch.float32):
    """Render a workload (optionally only its first ``n`` particles).

    Returns ``(refs [K,L,L], images [n,L,L], truth, blob_refs)`` in ``dtype``.
    """
    n = w.n if n is None else n
    refs64, blob = make_refs(w.K, w.L, w.blobs, w.sigma, w.amp, w.disc, w.seed_refs, device)
    imgs = torch.empty((n, w.L, w.L), dtype=dtype, device=device)
    truth = draw_particle_truth(n, w.K, int(w.shift_range), bool(w.mirror), w.seed_particles)
    render_particles(blob, truth, snr=w.snr, noise_seed=w.seed_noise, device=device, out=imgs)
    return refs64.to(dtype), imgs, truth, blob
