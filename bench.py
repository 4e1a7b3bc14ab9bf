"""Benchmark: multi-reference alignment throughput (images/s) on synthetic particles.

One step is the whole hot path over one stack: reference preparation
(polar + ring FFT of the K references), alignment of every particle at every
shift against every reference with and without mirror (polar resampling,
ring FFT, spectrum contraction, inverse angular FFT, argmax, pose decode)
and the class-average update.  The workload is the 100,000-particle,
76 x 76 px, K = 100, 81-shift stack (rings 1..35, mirror on); inputs (2.3 GB)
are larger than the 129 MB L2, so no flush is needed between steps.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
        [--precision fp32|bf16|fp16] [--n N_IMAGES]
Under torchrun each rank aligns its own stack (weak scaling); the class sums
are the one exchange step (all-reduce), then each rank finalises.
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "mra_n100k_L76_K100_shift4"
METRIC = "MRA images/s at stated K x shifts (BF16+rescore vs FP32 path)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
SM_COUNT_NOMINAL = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32-path comparison run")
    ap.add_argument("--n", type=int, default=None, help="override the stack size (testing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic workload (default: the 100,000-particle bench stack; the others are for "
                         "extra measurements, e.g. mra_n50k_L128_K200_shift6)")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests in each serving run (Poisson streams at 0.5, 0.7 and 0.9 x capacity); 0 skips it")
    ap.add_argument("--kernel", default="tuned", choices=["tuned", "mma_sync", "tcgen05"],
                    help="contraction kernel of the 16-bit M = 256 path: the autotuner's choice (default) or a fixed one")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the larger-box workload leg (128 px, K = 200, 169 shifts, three precisions)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# algorithmic work (per launch of the dominant kernel)
# ---------------------------------------------------------------------------

def path_work(info_M, rings):
    """FP32 flops per (row, reference) pair: contraction 8 sum_f R_f + inverse DFT 5 M log2 M."""
    M = info_M
    R = [sum(1 for _, n in rings if n // 2 >= f) for f in range(M // 2 + 1)]
    return 8 * sum(R), 5 * M * int(round(math.log2(M)))


def ring_table(r1, r2, dr):
    out = []
    for r in range(r1, r2 + 1, dr):
        n = 1
        while n < 2 * math.pi * r:
            n *= 2
        out.append((r, n))
    return out


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(self.rows), "reasons": reasons}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

def _oracle_worker(args):
    import numpy as np
    from oracle import mra_oracle as O
    imgs, refs, cfgd = args
    cfg = O.MRAConfig(**cfgd)
    spec = O.reference_spectra(refs, cfg)
    for im in imgs:
        O.align_one(im, spec, cfg)
    return len(imgs)


def cpu_baseline(w, n_sample, refs_np, imgs_np):
    """Time the oracle (as it stands) on n_sample images over a spawn pool of all host cores."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cfgd = dict(L=w.L, first_ring=w.first_ring, last_ring=w.last_ring, ring_step=w.ring_step,
                shift_range=w.shift_range, shift_step=w.shift_step, mirror=w.mirror)
    per = max(1, n_sample // cores)
    jobs = [(imgs_np[i:i + per], refs_np, cfgd) for i in range(0, n_sample, per)]
    env_keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes=min(cores, len(jobs))) as pool:
            pool.map(_oracle_worker, [(jobs[0][0][:1], refs_np, cfgd)] * min(cores, len(jobs)))  # warm imports
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_worker, jobs))
            dt = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": done / dt, "unit": "images/s", "cores": min(cores, len(jobs)), "kind": "oracle",
            "sample": f"{done} images of the {w.n}-image stack (K={w.K}, S={int(round(2 * w.shift_range / w.shift_step + 1)) ** 2}, mirror on), FP64 NumPy, one single-threaded worker per core",
            "seconds": dt}


# ---------------------------------------------------------------------------
# reference arm
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import synth
    w = synth.WORKLOADS[args.workload]
    # each step a bounded sample (one image per host core, 16 on the GPU machine), and every step a
    # different slice of a 400-image subset of the stack, so the timed steps together cover
    # hundreds of distinct images
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    sample = max(8, min(16, cores))
    pool_n = 400
    refs, imgs, _, _ = synth.make_workload(w, n=pool_n)
    refs_np = refs.double().numpy()
    imgs_np = imgs.double().numpy()
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * sample) % (pool_n - sample + 1)
        r = cpu_baseline(w, sample, refs_np, imgs_np[lo:lo + sample])
        if step >= args.warmup:
            times.append(r)
    value = statistics.mean(t["value"] for t in times)
    covered = min(pool_n, (args.warmup + args.steps) * sample)
    ms = 1000.0 * w.n / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": w.n, "L": w.L, "K": w.K,
                       "S": int(round(2 * w.shift_range / w.shift_step + 1)) ** 2,
                       "rings": f"{w.first_ring}..{w.last_ring}",
                       "mirror": 1, "path": "FP64 oracle (explicit DFT sums)",
                       "step": f"{sample} images per step (a different slice of a {pool_n}-image subset each "
                               f"step, {covered} distinct images over the run), scaled to the stack"},
            "cpu_baseline": {"value": value, "unit": "images/s", "cores": times[-1]["cores"], "kind": "oracle",
                             "sample": f"{covered} distinct images of the stack, {sample} per step; " + times[-1]["sample"]},
            "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2011_05755_gb300 as mra
    from paper_2011_05755_gb300.shard import allreduce_class_sums
    import synth
    w = synth.WORKLOADS[args.workload]
    n = args.n or w.n
    prec = {"fp32": mra.MRA_FP32, "bf16": mra.MRA_BF16_RESCORE, "fp16": mra.MRA_FP16_RESCORE}[args.precision]

    # CPU baseline first (spawned workers, before heavy GPU work), rank 0 at N = 1 only
    cpu_line = None
    refs_np = imgs_np = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the 200-image oracle subset of the stack (about 25 s on 16 host cores at 100 references and
        # 81 shifts); with rings beyond 40 (M = 512: the 128-pixel, 200-reference workload) an image
        # costs ~30x more and the sample is one image per core
        n_cpu = 200 if w.last_ring <= 40 else 16
        r64, i64, _, _ = synth.make_workload(w, n=n_cpu)
        refs_np, imgs_np = r64.double().numpy(), i64.double().numpy()
        cpu_line = cpu_baseline(w, n_cpu, refs_np, imgs_np)
        # the 500-image, K = 10, 25-shift workload, every image (about 2 s)
        w1 = synth.WORKLOADS["mra_n500_L76_K10_shift2"]
        r1, i1, _, _ = synth.make_workload(w1)
        full1 = cpu_baseline(w1, w1.n, r1.double().numpy(), i1.double().numpy())
        cpu_line["mra_n500_L76_K10_shift2"] = {k: full1[k] for k in ("value", "unit", "cores", "sample", "seconds")}

    # inputs: rank r renders its own particles (weak scaling)
    wr = synth.Workload(**{**w.__dict__, "seed_particles": w.seed_particles + 100 * rank,
                           "seed_noise": w.seed_noise + 100 * rank})
    refs, imgs, _, _ = synth.make_workload(wr, n=n, device=dev)
    K, L = w.K, w.L
    torch.cuda.synchronize()
    peaks = {}
    try:
        peaks = json.load(open(PEAKS_FILE))
    except Exception:
        pass
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    rings = ring_table(w.first_ring, w.last_ring, w.ring_step)
    stream = torch.cuda.current_stream()

    def run_path(prec_code, label, w, refs, imgs, n, steps, warmup, force_kernel=None):
        K, L = w.K, w.L
        rings = ring_table(w.first_ring, w.last_ring, w.ring_step)
        # launch choices of this configuration from the autotuner (timed candidates, cached in JSON)
        from paper_2011_05755_gb300.autotune import tune
        if force_kernel is not None:  # one kernel at the library's default chunking
            choice = {"kernel": force_kernel, "chunk_images": 0, "candidates": []}
        elif args.kernel == "tuned" or prec_code == mra.MRA_FP32:
            choice = tune(L, w.first_ring, w.last_ring, w.ring_step, w.shift_range, w.shift_step, w.mirror, prec_code,
                          K)
        else:  # a fixed kernel (profiling runs): the library's default chunking
            choice = {"kernel": {"mma_sync": mra.MRA_KERNEL_MMA_SYNC, "tcgen05": mra.MRA_KERNEL_TCGEN05}[args.kernel],
                      "chunk_images": 0, "candidates": []}
        al = mra.Aligner(L, w.first_ring, w.last_ring, w.ring_step, w.shift_range, w.shift_step, w.mirror,
                         prec_code, choice["chunk_images"], choice["kernel"])
        poses = torch.empty((n, 8), dtype=torch.int32, device=dev)
        avg = torch.zeros((K, L, L), dtype=torch.float32, device=dev)
        counts = torch.zeros((K,), dtype=torch.int32, device=dev)
        sums = torch.zeros((K, L, L), dtype=torch.float32, device=dev)
        comp = torch.zeros_like(sums)

        def step(eager=False):
            if world == 1 and not eager:
                # set_refs + align + class average as one CUDA graph launch (captured on the second call)
                mra.mra_run_graph(al.h, refs, imgs, poses, avg, counts, stream)
                return
            al.set_refs(refs, stream)
            al.align(imgs, poses, stream)
            if world == 1:
                mra.mra_average(al.h, imgs, poses, avg, counts, stream)
            else:
                sums.zero_()
                comp.zero_()
                counts.zero_()
                mra.mra_class_sums(al.h, imgs, poses, sums, comp, counts, stream)
                allreduce_class_sums(sums, comp, counts)
                mra.mra_average_finalize(al.h, sums, comp, counts, avg, stream)

        for _ in range(max(warmup, 2)):
            step()
        mra.mra_sync(al.h)
        info = al.info
        graph = world == 1 and mra.mra_graph_info(al.h)
        clocks = ClockSampler(local)
        clocks.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clk = clocks.stop()
        mra.mra_sync(al.h)
        ms_total = ev0.elapsed_time(ev1)
        # per-stage device times and kernel launches: one more step, eager, with stage timing on
        mra.mra_profile(al.h, True)
        step(eager=True)
        mra.mra_sync(al.h)
        prof = mra.mra_profile_read(al.h)
        mra.mra_profile(al.h, False)
        prof_steps = 1
        if world > 1:
            t = torch.tensor([ms_total], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_total = float(t.item())
        ms_step = ms_total / steps
        S = info["S"]
        f_con, f_ifft = path_work(info["M"], rings)
        sm_max = clk.get("sm_max_mhz") or 2070.0
        alu_peak = nsm * 128 * 2 * sm_max * 1e6 / 1e12
        alu_src = (f"FP32 FFMA: {nsm} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz (unit counts and max clock; "
                   "an FFMA probe measured 74.3 TFLOP/s)")
        # the kernel runs inside a step of about a second: the sustained (power-capped) peak applies
        tpeak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops", 1700.0)
        tsrc = ("bf16_tflops_sustained of MEASURED_PEAKS.json (cuBLAS bf16 GEMM looped for seconds under the "
                "power cap), of measured" if peaks.get("bf16_tflops_sustained") else
                "bf16_tflops of MEASURED_PEAKS.json (cuBLAS burst), of measured")

        def traffic_for(kernel, units):
            try:
                ent = json.load(open(TRAFFIC_FILE)).get(kernel)
                if ent and ent.get("source_hash") == source_hash(ent["sources"]):
                    return ent["bytes_per_unit"] * units
            except Exception:
                pass
            return None

        # the contraction / inverse-DFT kernel: one launch per chunk
        cc = prof["cc"]
        launches_cc = max(1, cc["launches"])
        pairs_per_launch = n * S * K * prof_steps / launches_cc
        cc_s = cc["ms"] / launches_cc / 1000.0
        if prec_code == mra.MRA_FP32:
            kname = "cc_fp32_kernel"
            flops = pairs_per_launch * (f_con + f_ifft)
            cc_line = {"bound": "alu", "kernel": kname + " (FP32 contraction + inverse angular DFT + argmax)",
                       "achieved": flops / cc_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s", "peak_source": alu_src}
        else:
            kname = {256: "cc_tc256_kernel", 512: "cc_tc512_kernel"}.get(info["M"], "cc_tc_kernel")
            if info["M"] == 256 and choice["kernel"] == mra.MRA_KERNEL_TCGEN05:
                kname = "cc_umma256_kernel"
            tc_idft = info["M"] in (256, 512)  # the inverse DFT on tensor cores too (M <= 128: FP32)
            flops = pairs_per_launch * (f_con + (f_ifft if tc_idft else 0))
            cc_line = {"bound": "tensor", "kernel": kname + " (16-bit tensor-core contraction"
                       + (" and inverse angular DFT" if tc_idft else " + FP32 inverse DFT") + ", row maxima)",
                       "achieved": flops / cc_s / 1e12, "peak": tpeak, "unit": "TFLOP/s", "peak_source": tsrc}
        cc_line.update({"frac": cc_line["achieved"] / cc_line["peak"], "traffic": traffic_for(kname, pairs_per_launch),
                        "unit_of_work": "(row, reference) pair", "flop_per_unit": flops / pairs_per_launch,
                        "units_per_launch": pairs_per_launch, "avg_launch_ms": cc_s * 1000.0,
                        "share_of_step": cc["ms"] / (prof_steps * ms_step)})
        # polar resampling + ring FFT: one launch per chunk (plus one for the references)
        po = prof["polar"]  # particle launches only (the references' launch is the "refs" stage)
        launches_po = max(1, po["launches"])
        rows_per_launch = n * S * prof_steps / launches_po
        po_s = po["ms"] / launches_po / 1000.0
        f_row = sum(2.5 * nr * math.log2(nr) + 9.0 * nr for _, nr in rings)
        po_line = {"bound": "alu", "kernel": "polar_fft_kernel (bilinear polar resampling + ring FFT)",
                   "achieved": rows_per_launch * f_row / po_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                   "peak_source": alu_src, "unit_of_work": "(image, shift) row", "flop_per_unit": f_row,
                   "units_per_launch": rows_per_launch, "avg_launch_ms": po_s * 1000.0,
                   "traffic": traffic_for("polar_fft_kernel", rows_per_launch),
                   "share_of_step": po["ms"] / (prof_steps * ms_step)}
        po_line["frac"] = po_line["achieved"] / po_line["peak"]
        roofline, other = (cc_line, po_line) if cc["ms"] >= po["ms"] else (po_line, cc_line)
        roofline = dict(roofline, other_kernel=other)
        # whole-step lower bound: each unit's algorithmic work at its peak
        pairs = n * S * K
        rows = n * S
        L2px = L * L * 4
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        half = prec_code != mra.MRA_FP32
        a_bytes = info["n_bins_padded"] * 8 if not half else sum(
            -(-sum(1 for _, nr in rings if nr // 2 >= f) // 16) for f in range(info["M"] // 2 + 1)) * 64
        tc_idft = info["M"] in (256, 512)
        t_tensor = pairs * (f_con + (f_ifft if tc_idft else 0)) / (tpeak * 1e12) if half else 0.0
        fp32_flops = rows * f_row                                   # polar resampling + ring FFTs
        if not half:
            fp32_flops += pairs * (f_con + f_ifft)                  # FP32 contraction + inverse DFT
        else:
            if not tc_idft:
                fp32_flops += pairs * f_ifft                        # FP32 inverse DFT of the 16-bit path
            fp32_flops += n * 8 * (f_row + f_con + f_ifft)          # rescore of 8 rows per image
        t_fp32 = fp32_flops / (alu_peak * 1e12)
        hbm_bytes = 2 * n * L2px + 2 * rows * a_bytes + (pairs * 16 if half else 0)
        t_hbm = hbm_bytes / (hbm_peak * 1e9)
        bound_ms = 1000.0 * max(t_tensor, t_fp32, t_hbm)
        step_roof = {"t_tensor_ms": 1000.0 * t_tensor, "t_fp32_ms": 1000.0 * t_fp32, "t_hbm_ms": 1000.0 * t_hbm,
                     "bound_ms": bound_ms, "ms_per_step": ms_step, "frac": bound_ms / ms_step,
                     "note": "each unit's algorithmic work per step at its peak (tensor: contraction and, for "
                             "M = 256 and 512, inverse-DFT flops at the sustained BF16 peak; FP32: polar rows, "
                             "FP32 contraction / "
                             "inverse DFT and the 8 rescored rows per image; HBM: stack read twice, spectra "
                             "written and read once, row maxima); frac = the largest / measured step time"}
        launches_step = sum(v["launches"] for v in prof.values())
        return {"label": label, "al": al, "value": n * world / (ms_step / 1000.0), "ms_step": ms_step,
                "prof": prof, "roofline": roofline, "clocks": clk, "info": info, "step_roofline": step_roof,
                "gpu_launches": launches_step * steps,
                "launch": {"graph": bool(graph), "graph_launches_per_step": 1 if graph else 0,
                           "kernel_launches_per_step": launches_step,
                           "tuned": {"kernel": {0: "default", 1: "mma.sync", 2: "tcgen05"}[choice["kernel"]],
                                     "chunk_images": choice["chunk_images"], "chunk_used": info["chunk_images"],
                                     "candidates": choice["candidates"]}}}

    prec_label = args.precision
    main_res = run_path(prec, prec_label, w, refs, imgs, n, args.steps, args.warmup)
    cmp_res = None
    if not args.no_compare and prec != mra.MRA_FP32:
        cmp_res = run_path(mra.MRA_FP32, "fp32", w, refs, imgs, n, args.steps, args.warmup)
        cmp_res["al"].close()
    # the same 16-bit step on the tcgen05 contraction kernel (M = 256 only), its own roofline
    umma_res = None
    if (not args.no_compare and prec != mra.MRA_FP32 and world == 1 and
            max(nr for _, nr in ring_table(w.first_ring, w.last_ring, w.ring_step)) == 256):
        umma_res = run_path(prec, "tcgen05", w, refs, imgs, n, 2, 2, force_kernel=mra.MRA_KERNEL_TCGEN05)
        umma_res["al"].close()
    al = main_res["al"]
    value, ms_step, prof, roofline, clk, info = (main_res[k] for k in ("value", "ms_step", "prof", "roofline",
                                                                        "clocks", "info"))
    S = info["S"]
    gpu_launches = main_res["gpu_launches"]
    launch = main_res["launch"]

    # end to end through the host-buffer entry point (pinned memory, copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        h_refs = refs.cpu().pin_memory()
        h_imgs = imgs.cpu().pin_memory()
        h_poses = torch.empty((n, 8), dtype=torch.int32).pin_memory()
        h_avg = torch.zeros((K, L, L), dtype=torch.float32).pin_memory()
        h_cnt = torch.zeros((K,), dtype=torch.int32).pin_memory()
        mra.mra_run_host(al.h, h_refs, h_imgs, h_poses, h_avg, h_cnt, stream)  # warm
        reps = max(1, min(3, args.steps))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            mra.mra_run_host(al.h, h_refs, h_imgs, h_poses, h_avg, h_cnt, stream)
        dt = (time.perf_counter() - t0) / reps
        if world > 1:
            t = torch.tensor([dt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": n * world / dt, "unit": "images/s",
               "h2d_bytes_per_step": (h_refs.numel() + h_imgs.numel()) * 4,
               "d2h_bytes_per_step": h_poses.numel() * 4 + h_avg.numel() * 4 + h_cnt.numel() * 4,
               "ms_per_step": dt * 1000.0, "api": "mra_run_host"}

    # the larger-box workload (128 x 128 px, K = 200, 169 shifts, rings 1..60, M = 512) in all three
    # precisions: a 10,000-image stack, 3 timed steps each
    larger_box = None
    if rank == 0 and world == 1 and not args.no_extra:
        w3 = synth.WORKLOADS["mra_n50k_L128_K200_shift6"]
        n3 = 10000
        refs3, imgs3, _, _ = synth.make_workload(w3, n=n3, device=dev)
        larger_box = {"workload": w3.name, "n_images": n3, "steps": 3, "warmup": 2,
                      "note": "the 50,000-image workload's shapes on a 10,000-image stack (images/s does not "
                              "depend on the stack size once it spans many chunks)"}
        for pl, pc in (("bf16", mra.MRA_BF16_RESCORE), ("fp16", mra.MRA_FP16_RESCORE), ("fp32", mra.MRA_FP32)):
            r3 = run_path(pc, pl, w3, refs3, imgs3, n3, 3, 2)
            larger_box[pl] = {"value": r3["value"], "unit": "images/s", "ms_per_step": r3["ms_step"],
                              "roofline": r3["roofline"], "clocks": r3["clocks"], "launch": r3["launch"],
                              "stages": r3["prof"], "gpu_launches": r3["gpu_launches"]}
            r3["al"].close()
        del refs3, imgs3
        torch.cuda.empty_cache()

    serving = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        from paper_2011_05755_gb300.serve import run_stream
        al.close()  # the stream run holds its own handles
        del imgs
        torch.cuda.empty_cache()
        serving = run_stream(args.serve_requests, [0.5, 0.7, 0.9], prec, calibration_requests=24)
        serving["precision"] = args.precision

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16+f32", "fp16": "f16+f32"}[args.precision],
            "data": "synthetic (seeded Gaussian-blob references and particles, SNR 0.1)",
            "config": {"workload": args.workload, "n_per_gpu": n, "L": L, "K": K, "S": S,
                       "rings": f"{w.first_ring}..{w.last_ring}", "M": info["M"],
                       "mirror": 1, "path": {"fp32": "FP32", "bf16": "BF16 contraction + FP32 rescore of top-8 rows",
                                             "fp16": "FP16 contraction + FP32 rescore of top-8 rows"}[args.precision],
                       "step": "set_refs + align + class average",
                       "l2": f"inputs ({n * L * L * 4 / 1e9:.1f} GB/GPU) larger than L2; no flush"},
            "e2e": e2e, "gpu_launches": gpu_launches, "launch": launch, "stages": prof, "roofline": roofline,
            "cpu_baseline": cpu_line, "clocks": clk, "serving": serving, "larger_box": larger_box,
            "step_roofline": main_res["step_roofline"],
        }
        if cmp_res is not None:
            line["fp32_path"] = {"value": cmp_res["value"], "ms_per_step": cmp_res["ms_step"],
                                 "speedup_of_headline_path": value / cmp_res["value"],
                                 "roofline": cmp_res["roofline"], "stages": cmp_res["prof"],
                                 "gpu_launches": cmp_res["gpu_launches"], "launch": cmp_res["launch"],
                                 "clocks": cmp_res["clocks"],
                                 "step_roofline": cmp_res["step_roofline"]}
        if umma_res is not None:
            line["tcgen05_path"] = {"value": umma_res["value"], "ms_per_step": umma_res["ms_step"], "steps": 2,
                                    "relative_to_headline_path": umma_res["value"] / value,
                                    "roofline": umma_res["roofline"], "stages": umma_res["prof"],
                                    "gpu_launches": umma_res["gpu_launches"], "launch": umma_res["launch"],
                                    "clocks": umma_res["clocks"],
                                    "note": "the headline step with the tcgen05 / TMEM contraction kernel "
                                            "(MRA_KERNEL_TCGEN05) at the library's default chunk; the autotuner "
                                            "keeps mma.sync for the headline where it is faster"}
        print(json.dumps(line), flush=True)
    al.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
