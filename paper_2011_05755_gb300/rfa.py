"""Reference-free alignment (RFA): every particle against one common reference.

RFA is the single-reference case of the multi-reference search (Sec. 3: the
MRA kernels differ from RFA only in correlating each particle with all K
references instead of one).  The reference is built from the data: it starts
as the unaligned mean of the stack, and each pass aligns every particle
against it (polar resampling at every shift, ring FFTs, contraction,
inverse angular DFT, argmax) and replaces it by the normalised average of
the aligned particles, until fewer than ``tol`` of the particles change pose.
Every arithmetic step runs in the library's kernels (``mra_align``,
``mra_average``, ``mra_refresh_refs``) with K = 1.

CLI (the paper's RFA timing sweep, Fig. 3(b): computation time against the
shift search range; synthetic 90 x 90 px particles, particle radius 36 px):

    python -m paper_2011_05755_gb300.rfa [--n 20000] [--ranges 1 2 3 4 5 6] [--precision fp32]
"""
from __future__ import annotations

import argparse
import json
from typing import Optional

import numpy as np
import torch

from . import (MRA_BF16_RESCORE, MRA_FP16_RESCORE, MRA_FP32, Aligner, decode_poses, mra_average, mra_refresh_refs,
               mra_sync)


def unaligned_mean(al: Aligner, imgs: torch.Tensor) -> torch.Tensor:
    """Normalised mean of the stack with no alignment (the usual RFA start), [L, L]."""
    n, L = imgs.shape[0], imgs.shape[-1]
    ref = torch.zeros((1, L, L), dtype=torch.float32, device=imgs.device)
    al.set_refs(ref)  # K = 1 for the averaging
    poses = torch.zeros((n, 8), dtype=torch.int32, device=imgs.device)
    counts = torch.zeros((1,), dtype=torch.int32, device=imgs.device)
    mra_average(al.h, imgs, poses, ref, counts)
    mra_refresh_refs(al.h, ref, counts)
    return ref[0]


def rfa(imgs: torch.Tensor, cfg: dict, n_iter: int = 10, tol: float = 1e-3, precision: int = MRA_FP32,
        ref0: Optional[torch.Tensor] = None) -> dict:
    """Iterate align -> average -> normalise with one reference.

    ``cfg``: dict with L, first_ring, last_ring, ring_step, shift_range,
    shift_step, mirror.  Returns ``{"ref" [L, L], "poses" [n, 8], "history"}``;
    a pass's ``changed`` is the fraction of particles whose (angle, shift,
    mirror) differs from the previous pass.
    """
    n, L = imgs.shape[0], imgs.shape[-1]
    al = Aligner(cfg["L"], cfg["first_ring"], cfg["last_ring"], cfg.get("ring_step", 1), cfg.get("shift_range", 0.0),
                 cfg.get("shift_step", 1.0), cfg.get("mirror", 1), precision)
    ref = (unaligned_mean(al, imgs) if ref0 is None else ref0.to(imgs.device, torch.float32)).contiguous()
    poses = torch.zeros((n, 8), dtype=torch.int32, device=imgs.device)
    stream = torch.cuda.current_stream()
    prev = None
    history = []
    for it in range(n_iter):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        refs = ref[None].contiguous()
        al.set_refs(refs, stream)
        al.align(imgs, poses, stream)
        new = refs.clone()
        counts = torch.zeros((1,), dtype=torch.int32, device=imgs.device)
        mra_average(al.h, imgs, poses, new, counts, stream)
        mra_refresh_refs(al.h, new, counts, None, None, stream)
        e1.record(stream)
        mra_sync(al.h, stream)
        ms = e0.elapsed_time(e1)
        p = poses[:, 1:4].cpu().numpy().copy()  # ang_idx, mirror, shift_idx
        changed = 1.0 if prev is None else float(np.mean(np.any(p != prev, axis=1)))
        prev = p
        ref = new[0]
        history.append({"iteration": it, "changed": changed, "ms": ms, "images_per_s": n / (ms / 1000.0)})
        if changed < tol:
            break
    al.close()
    return {"ref": ref, "poses": poses, "history": history}


def _main():
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--ranges", type=int, nargs="+", default=[1, 2, 3, 4, 5, 6])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    prec = {"fp32": MRA_FP32, "bf16": MRA_BF16_RESCORE, "fp16": MRA_FP16_RESCORE}[args.precision]
    dev = torch.device("cuda", 0)
    L, r2 = 90, 36
    refs, blob = synth.make_refs(1, L, blobs=20, sigma=(3.5, 9.5), disc=33.0, seed=1006)
    out = {"workload": f"RFA sweep: n={args.n}, L={L}, rings 1..{r2}, K=1, SNR 0.1, mirror on", "precision": args.precision,
           "ranges": {}}
    for R in args.ranges:
        imgs, _ = synth.make_particles(blob, args.n, shift_range=R, mirror=True, snr=0.1, seed=2006, noise_seed=3006,
                                       device=dev)
        imgs = imgs.float().contiguous()
        al = Aligner(L, 1, r2, 1, float(R), 1.0, 1, prec)
        al.set_refs(refs.float().to(dev))
        poses = torch.empty((args.n, 8), dtype=torch.int32, device=dev)
        avg = torch.zeros((1, L, L), dtype=torch.float32, device=dev)
        cnt = torch.zeros((1,), dtype=torch.int32, device=dev)
        for _ in range(2):
            al.align(imgs, poses)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            al.align(imgs, poses)
            mra_average(al.h, imgs, poses, avg, cnt)
        e1.record()
        mra_sync(al.h)
        ms = e0.elapsed_time(e1) / args.reps
        S = (2 * R + 1) ** 2
        out["ranges"][str(R)] = {"shifts": S, "ms_per_pass": ms, "images_per_s": args.n / (ms / 1000.0)}
        al.close()
        del imgs
    print(json.dumps(out))


if __name__ == "__main__":
    _main()
