"""Launch-parameter tuning per configuration, cached in JSON.

The library exposes two launch choices per handle (``mra_config_t``):

* ``kernel``: for the 16-bit paths at M = 256, the warp-level mma.sync
  kernel (tiles of 8 rows x 8 references, two CTAs per SM) or the tcgen05
  kernel (tiles of 16 rows x 8 references, TMEM accumulators, one persistent
  CTA per SM);
* ``chunk_images``: images per internal chunk (the particle spectra of one
  chunk are the largest workspace; fewer, larger chunks mean fewer launches
  and kernel tails, smaller ones a smaller footprint).  Candidates: the
  library's default (a 2 GiB workspace, rounded to whole rescore waves),
  1,024 images, and three times the default.

:func:`tune` times every candidate on a synthetic stack of the
configuration's shape (the alignment's work does not depend on the pixel
values) with CUDA events and keeps the fastest.  Results are cached per
(device, L, rings, shift grid, mirror, precision, K) in a JSON file
(``MRA_TUNE_CACHE`` or ``~/.cache/mra_gb300/tune.json``), so a configuration
is tuned once per machine.  :func:`tuned_aligner` builds an
:class:`~paper_2011_05755_gb300.Aligner` with the tuned choice.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

import torch

from . import (MRA_FP32, MRA_KERNEL_AUTO, MRA_KERNEL_MMA_SYNC, MRA_KERNEL_TCGEN05, Aligner, mra_sync)

__all__ = ["tune", "tuned_aligner", "cache_path", "candidates"]


def cache_path() -> str:
    return os.environ.get("MRA_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "mra_gb300",
                                                            "tune.json")


def _ring_M(first_ring: int, last_ring: int, ring_step: int) -> int:
    r = first_ring + (last_ring - first_ring) // ring_step * ring_step
    n = 1
    while n < 2 * math.pi * r:
        n *= 2
    return n


def candidates(first_ring: int, last_ring: int, ring_step: int, precision: int) -> list:
    """The (kernel, chunk_images) pairs worth timing for a configuration."""
    kernels = [MRA_KERNEL_AUTO]
    if precision != MRA_FP32 and _ring_M(first_ring, last_ring, ring_step) == 256:
        kernels = [MRA_KERNEL_MMA_SYNC, MRA_KERNEL_TCGEN05]
    chunks = [0, 1024]  # 0: sized from the library's 2 GiB workspace budget
    return [(k, c) for k in kernels for c in chunks]


def _key(dev, L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, precision, K) -> str:
    name = torch.cuda.get_device_name(dev).replace(" ", "_")
    return (f"{name}|L{L}|r{first_ring}-{last_ring}-{ring_step}|s{shift_range:g}/{shift_step:g}|m{mirror}"
            f"|p{precision}|K{K}")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(L: int, first_ring: int, last_ring: int, ring_step: int = 1, shift_range: float = 0.0,
         shift_step: float = 1.0, mirror: int = 1, precision: int = MRA_FP32, K: int = 8,
         n_probe: Optional[int] = None, reps: int = 3, device=None, cache: Optional[str] = None,
         refresh: bool = False) -> dict:
    """The fastest launch choice for a configuration: ``{"kernel", "chunk_images", "ms_per_image",
    "candidates": [...]}`` (from the cache unless ``refresh``)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    path = cache or cache_path()
    key = _key(dev, L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, precision, K)
    db = _load(path)
    if key in db and not refresh:
        return db[key]
    nx = int(round(2 * shift_range / shift_step)) + 1
    S = nx * nx
    if n_probe is None:  # about 4e8 (row, reference) pairs: several chunks of the default size
        n_probe = int(min(8192, max(256, 4e8 / (S * K))))
    g = torch.Generator(device=dev).manual_seed(1234)
    refs = torch.randn((K, L, L), generator=g, device=dev)
    imgs = torch.randn((n_probe, L, L), generator=g, device=dev)
    poses = torch.empty((n_probe, 8), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    results = []
    todo = list(candidates(first_ring, last_ring, ring_step, precision))
    while todo:
        kernel, chunk = todo.pop(0)
        al = Aligner(L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, precision, chunk, kernel)
        try:
            al.set_refs(refs, stream)
            al.align(imgs, poses, stream)  # warm-up: workspaces and kernel attributes
            mra_sync(al.h, stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                al.align(imgs, poses, stream)
            e1.record(stream)
            mra_sync(al.h, stream)
            ms = e0.elapsed_time(e1) / reps
            used = al.info["chunk_images"]
            results.append({"kernel": kernel, "chunk_images": chunk, "ms_per_image": ms / n_probe,
                            "chunk_used": used})
            if chunk == 0 and 3 * used < n_probe:  # three default chunks in one (whole waves stay whole)
                todo.append((kernel, 3 * used))
        finally:
            al.close()
    best = min(results, key=lambda r: r["ms_per_image"])
    out = {"kernel": best["kernel"], "chunk_images": best["chunk_images"], "ms_per_image": best["ms_per_image"],
           "n_probe": n_probe, "candidates": results}
    db = _load(path)
    db[key] = out
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return out


def tuned_aligner(L: int, first_ring: int, last_ring: int, ring_step: int = 1, shift_range: float = 0.0,
                  shift_step: float = 1.0, mirror: int = 1, precision: int = MRA_FP32, K: int = 8, **kw):
    """An Aligner with the tuned (kernel, chunk_images) of the configuration; returns (aligner, choice)."""
    choice = tune(L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, precision, K, **kw)
    al = Aligner(L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, precision,
                 choice["chunk_images"], choice["kernel"])
    return al, choice
