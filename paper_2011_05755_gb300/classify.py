"""Iterative 2D classification by multi-reference alignment.

The outer loop of Alg. 1 (its convergence loop): align every
particle against the current references, rebuild the class averages from
the aligned images, normalise them (zero mean, unit standard deviation over
the box) and use them as the next references (Sec. 2 describes the same
classification outline).  A class that received no particle is reseeded with
a randomly chosen particle.  The loop stops after ``n_iter`` passes or when
fewer than ``tol`` of the particles changed class.  Every arithmetic step
runs in the library's kernels (``mra_align``, ``mra_average``,
``mra_refresh_refs``); this module only sequences them, keeps the small
host-side bookkeeping (changed-assignment fraction, reseed choice) and
writes checkpoints.

CLI (synthetic 200,000-particle, K = 500 workload; compares the BF16+rescore
and FP32 paths):

    python -m paper_2011_05755_gb300.classify [--n N] [--K K] [--iters 10] [--precision bf16] [--compare]
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Optional

import numpy as np
import torch

from . import (MRA_BF16_RESCORE, MRA_FP16_RESCORE, MRA_FP32, Aligner, decode_poses, mra_average, mra_refresh_refs,
               mra_sync)


def identity_poses(labels: torch.Tensor) -> torch.Tensor:
    """mra_pose_t rows with class `labels`, no shift, no rotation, no mirror (int32 [n, 8])."""
    n = labels.shape[0]
    p = torch.zeros((n, 8), dtype=torch.int32, device=labels.device)
    p[:, 0] = labels.to(torch.int32)
    return p


def initial_references(al: Aligner, imgs: torch.Tensor, K: int, seed: int) -> torch.Tensor:
    """Unaligned class means of a random equal partition of the particles, normalised."""
    n = imgs.shape[0]
    rng = np.random.default_rng(seed)
    labels = torch.from_numpy((rng.permutation(n) % K).astype(np.int32)).to(imgs.device)
    refs = torch.zeros((K, imgs.shape[1], imgs.shape[2]), dtype=torch.float32, device=imgs.device)
    counts = torch.zeros((K,), dtype=torch.int32, device=imgs.device)
    al.set_refs(refs)  # the class count of the averaging comes from the reference set
    mra_average(al.h, imgs, identity_poses(labels), refs, counts)
    mra_refresh_refs(al.h, refs, counts)
    return refs


def classify(imgs: torch.Tensor, refs0: torch.Tensor, cfg: dict, n_iter: int = 10, tol: float = 1e-3,
             precision: int = MRA_FP32, seed: int = 0, checkpoint_dir: Optional[str] = None,
             resume: bool = False) -> dict:
    """Run the classification loop; returns ``{"refs", "poses", "history"}``.

    ``cfg``: dict with L, first_ring, last_ring, ring_step, shift_range,
    shift_step, mirror.  With ``checkpoint_dir`` the references, poses and the
    iteration number are saved as .npy after every pass; ``resume`` restarts
    from the last saved pass.
    """
    n, L = imgs.shape[0], imgs.shape[-1]
    K = refs0.shape[0]
    al = Aligner(cfg["L"], cfg["first_ring"], cfg["last_ring"], cfg.get("ring_step", 1), cfg.get("shift_range", 0.0),
                 cfg.get("shift_step", 1.0), cfg.get("mirror", 1), precision)
    refs = refs0.clone().contiguous()
    poses = torch.zeros((n, 8), dtype=torch.int32, device=imgs.device)
    prev = None
    start = 0
    history = []
    rng = np.random.default_rng(seed)
    if resume and checkpoint_dir and os.path.exists(os.path.join(checkpoint_dir, "iteration.npy")):
        start = int(np.load(os.path.join(checkpoint_dir, "iteration.npy"))) + 1
        refs = torch.from_numpy(np.load(os.path.join(checkpoint_dir, "refs.npy"))).to(imgs.device).contiguous()
        poses = torch.from_numpy(np.load(os.path.join(checkpoint_dir, "poses.npy"))).to(imgs.device).contiguous()
        prev = poses[:, 0].cpu().numpy().copy()
        rng = np.random.default_rng([seed, start])
        history = json.load(open(os.path.join(checkpoint_dir, "history.json")))
    stream = torch.cuda.current_stream()
    for it in range(start, n_iter):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        al.set_refs(refs, stream)
        al.align(imgs, poses, stream)
        new_refs = refs.clone()  # classes that stay empty keep their reference until reseeded
        counts = torch.zeros((K,), dtype=torch.int32, device=imgs.device)
        mra_average(al.h, imgs, poses, new_refs, counts, stream)
        counts_h = counts.cpu().numpy()
        empty = np.flatnonzero(counts_h == 0)
        reseed = None
        if empty.size:
            rs = np.full(K, -1, dtype=np.int32)
            rs[empty] = rng.integers(0, n, size=empty.size)
            reseed = torch.from_numpy(rs).to(imgs.device)
        mra_refresh_refs(al.h, new_refs, counts, reseed, imgs if reseed is not None else None, stream)
        e1.record(stream)
        mra_sync(al.h, stream)
        ms = e0.elapsed_time(e1)
        k_now = poses[:, 0].cpu().numpy().copy()
        changed = 1.0 if prev is None else float(np.mean(k_now != prev))
        prev = k_now
        refs = new_refs
        history.append({"iteration": it, "changed": changed, "empty_classes": int(empty.size), "ms": ms,
                        "images_per_s": n / (ms / 1000.0)})
        rng = np.random.default_rng([seed, it + 1])
        if checkpoint_dir:
            os.makedirs(checkpoint_dir, exist_ok=True)
            np.save(os.path.join(checkpoint_dir, "refs.npy"), refs.cpu().numpy())
            np.save(os.path.join(checkpoint_dir, "poses.npy"), poses.cpu().numpy())
            np.save(os.path.join(checkpoint_dir, "iteration.npy"), np.array(it))
            json.dump(history, open(os.path.join(checkpoint_dir, "history.json"), "w"))
        if changed < tol:
            break
    al.close()
    return {"refs": refs, "poses": poses, "history": history}


def adjusted_rand_index(a: np.ndarray, b: np.ndarray) -> float:
    """Adjusted Rand index of two labelings (Hubert and Arabie)."""
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    table = np.zeros((ai.max() + 1, bi.max() + 1), dtype=np.int64)
    np.add.at(table, (ai, bi), 1)

    def comb2(x):
        x = x.astype(np.float64)
        return x * (x - 1) / 2.0

    sum_ij = comb2(table).sum()
    sum_a = comb2(table.sum(axis=1)).sum()
    sum_b = comb2(table.sum(axis=0)).sum()
    n = comb2(np.array(a.size)).item()
    expected = sum_a * sum_b / n if n else 0.0
    maxv = (sum_a + sum_b) / 2.0
    return float((sum_ij - expected) / (maxv - expected)) if maxv != expected else 1.0


def _main():
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--K", type=int, default=500)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--compare", action="store_true", help="also run the FP32 path and compare")
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    w = synth.Workload("mra_n200k_L76_K500_shift3_iter10", args.n, 76, args.K, 20, (3.0, 8.0), (0.5, 1.5), 28.0, 0.1,
                       1, 35, 1, 3.0, 1.0, 1, 1005, 2005, 3005)
    truth_refs, imgs, truth, _ = synth.make_workload(w, device=dev)
    cfg = dict(L=w.L, first_ring=w.first_ring, last_ring=w.last_ring, ring_step=1, shift_range=w.shift_range,
               shift_step=w.shift_step, mirror=1)
    init = Aligner(w.L, 1, 35, 1, w.shift_range, 1.0, 1)
    refs0 = initial_references(init, imgs, args.K, seed=7)
    init.close()
    prec = {"fp32": MRA_FP32, "bf16": MRA_BF16_RESCORE, "fp16": MRA_FP16_RESCORE}[args.precision]
    runs = {args.precision: classify(imgs, refs0, cfg, args.iters, 0.0, prec, seed=11)}
    if args.compare and args.precision != "fp32":
        runs["fp32"] = classify(imgs, refs0, cfg, args.iters, 0.0, MRA_FP32, seed=11)
    report = {"workload": w.name, "n": args.n, "K": args.K, "iterations": args.iters}
    for name, r in runs.items():
        p = decode_poses(r["poses"])
        report[name] = {"history": r["history"], "ari_vs_truth": adjusted_rand_index(p["k"], truth.k)}
    if args.compare and args.precision != "fp32":
        # one pass of both paths from the same references: the precision split alone
        for label, refs in (("initial_refs", refs0), ("final_fp32_refs", runs["fp32"]["refs"])):
            got = {}
            for name, code in ((args.precision, prec), ("fp32", MRA_FP32)):
                al = Aligner(w.L, 1, 35, 1, w.shift_range, 1.0, 1, code)
                al.set_refs(refs)
                got[name] = decode_poses(al.align(imgs))
                al.close()
            a, b = got[args.precision], got["fp32"]
            same_k = a["k"] == b["k"]
            same_pose = same_k & (a["ang_idx"] == b["ang_idx"]) & (a["shift_idx"] == b["shift_idx"]) & (
                a["mirror"] == b["mirror"])
            report["same_refs_" + label] = {"class": float(np.mean(same_k)), "pose": float(np.mean(same_pose)),
                                            "cc_rel_diff_median": float(np.median(np.abs(a["cc"] - b["cc"]) /
                                                                                  np.maximum(np.abs(b["cc"]), 1e-30)))}
    if "fp32" in runs and len(runs) == 2:
        a = decode_poses(runs[args.precision]["poses"])
        b = decode_poses(runs["fp32"]["poses"])
        same_class = a["k"] == b["k"]
        report["agreement_after_independent_runs"] = {
            "class": float(np.mean(same_class)),
            "ari_between_paths": adjusted_rand_index(a["k"], b["k"]),
            "pose_given_class": float(np.mean((a["ang_idx"] == b["ang_idx"]) & (a["shift_idx"] == b["shift_idx"])
                                              & (a["mirror"] == b["mirror"]) & same_class) / max(1e-12, np.mean(same_class))),
        }
    print(json.dumps(report))


if __name__ == "__main__":
    _main()
