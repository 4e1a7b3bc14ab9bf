"""The FP64 oracle over many images in a process pool (test helper).

Full-size parity samples (hundreds of images at 100 references and 81
shifts) take seconds of oracle time per image, so the tables are computed
by worker processes started with ``spawn`` (a pool forked after the CUDA
context exists would hang).  Each worker returns, per image, the oracle's
pose (argmax with the tie rule), its runner-up gap and the ``top`` largest
entries of the table with their indices, enough to assess a GPU pose that
differs from the oracle's in a near tie without shipping whole tables.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _worker(args):
    imgs, refs, cfgd, top = args
    from oracle import mra_oracle as O
    cfg = O.MRAConfig(**cfgd)
    spec = O.reference_spectra(refs, cfg)
    out = []
    for im in imgs:
        tab = O.cc_table(im, spec, cfg)
        p = O._pose_from_table(tab, cfg)
        flat = tab.ravel()
        idx = np.argpartition(flat, -top)[-top:]
        out.append(dict(k=p.k, shift_idx=p.shift_idx, mirror=p.mirror, ang_idx=p.ang_idx, cc=p.cc,
                        rel_gap=p.rel_gap, shape=tab.shape, top_idx=idx.astype(np.int64), top_val=flat[idx]))
    return out


def oracle_poses(imgs: np.ndarray, refs: np.ndarray, cfgd: dict, top: int = 64, procs: int | None = None):
    """Oracle poses of imgs [n, L, L] (FP64) against refs [K, L, L]; one dict per image."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    procs = max(1, min(procs or cores, len(imgs)))
    per = -(-len(imgs) // procs)
    jobs = [(imgs[i:i + per], refs, cfgd, top) for i in range(0, len(imgs), per)]
    env = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(processes=len(jobs)) as pool:
            parts = pool.map(_worker, jobs)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [p for part in parts for p in part]


def table_value(entry: dict, pose: tuple):
    """The oracle's table value at pose (k, shift_idx, mirror, ang_idx) if it is among the stored top
    entries, else None (the pose is then far from optimal)."""
    flat = int(np.ravel_multi_index(pose, entry["shape"]))
    hit = np.nonzero(entry["top_idx"] == flat)[0]
    return float(entry["top_val"][hit[0]]) if len(hit) else None
