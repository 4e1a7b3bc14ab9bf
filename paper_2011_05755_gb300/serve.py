"""Serving loop: continuous batching of particle-stack alignment requests.

Requests are particle stacks of uneven size and box size, each to be aligned
(Algorithm 1's per-image search) against a reference set that stays resident
on the device, one set per (L, K).  The loop

* admits arrived requests in arrival order while a slot is free and the
  stack fits the device-memory budget (a request larger than the whole budget
  is rejected with an error, never queued forever);
* serves a request in parts of at most ``part_images`` images, so that a
  large request's parts run on several slots at once (or, with
  ``requeue="back"``, so that small requests are served between them);
* batches: the admitted head part takes along later queued parts with the
  same (L, K), up to ``max_batch_images`` images, into one contiguous
  device stack and one ``mra_align`` call (images are independent, so a
  request's poses do not depend on how it was split or batched);
* overlaps: every slot owns a CUDA stream and, per box size, a library handle
  with its own workspace; the reference spectra are transformed once per set
  and copied into a slot's handle on the device when the slot switches sets
  (``mra_copy_refs``), so batches for different sets run side by side;
* is continuous: a slot is refilled the moment its batch completes, while the
  other slots keep running; new arrivals join the queue at any time.

Latency is completion minus arrival on the host clock (the host→device copy
of the stack and the device→host copy of the poses are inside it).

The scheduling policy (:class:`Scheduler`) is plain host code with no GPU
dependency; :class:`GpuExecutor` runs its batches through the library.

CLI (synthetic stream: 2,000 requests, sizes log-uniform on [200, 20000],
L in {64, 76, 96, 128}, K in {50, 100, 200}, shifts +-3 step 1, mirror on;
rings 1..L/2-4; Poisson arrivals at a fraction of the capacity measured in a
calibration pass):

    python -m paper_2011_05755_gb300.serve [--requests 2000] [--load 0.7 0.5 0.9] [--precision bf16]
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import json
import math
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

POSE_BYTES = 32


@dataclasses.dataclass
class Request:
    rid: int
    L: int
    K: int
    n: int
    arrival: float                              # seconds on the server clock
    imgs: Optional[torch.Tensor] = None         # host [n, L, L] float32 (pinned for overlap)
    admitted: float = math.nan
    done: float = math.nan
    poses: Optional[torch.Tensor] = None        # host int32 [n, 8] (mra_pose_t rows)
    error: str = ""
    batch_id: int = -1
    parts_left: int = 0                         # parts issued or queued and not yet finished
    next_off: int = 0                           # first image not yet given to a part

    @property
    def key(self) -> Tuple[int, int]:
        return (self.L, self.K)

    @property
    def device_bytes(self) -> int:
        return self.n * (self.L * self.L * 4 + POSE_BYTES)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclasses.dataclass
class Part:
    """Images [off, off + n) of one request: the unit the scheduler batches."""
    req: Request
    off: int
    n: int

    @property
    def key(self) -> Tuple[int, int]:
        return self.req.key

    @property
    def device_bytes(self) -> int:
        return self.n * (self.req.L * self.req.L * 4 + POSE_BYTES)


class Scheduler:
    """Admission and batching policy over request parts.

    The head of the queue is admitted first (FIFO, no overtaking while it
    waits for memory); queued parts with the same (L, K) are batched in up to
    ``max_batch_images``.  With ``part_images`` > 0 a request is served in
    parts of at most that many images; when a part is issued the request's
    next part is queued at the front (``requeue="front"``: the parts of a
    large request spread over the free slots and it finishes sooner) or at
    the back (``"back"``: round robin, small requests are served between the
    parts of a large one); 0 serves every request as one part.
    """

    def __init__(self, hbm_budget: int, n_slots: int, max_batch_images: int, part_images: int = 0,
                 requeue: str = "front"):
        if n_slots < 1 or hbm_budget <= 0 or max_batch_images < 1 or part_images < 0:
            raise ValueError("n_slots, hbm_budget and max_batch_images must be positive, part_images >= 0")
        if requeue not in ("front", "back"):
            raise ValueError("requeue must be 'front' or 'back'")
        self.requeue = requeue
        self.hbm_budget = int(hbm_budget)
        self.free_bytes = int(hbm_budget)
        self.free_slots = list(range(n_slots))
        self.max_batch_images = int(max_batch_images)
        self.part_images = int(part_images)
        self.queue: collections.deque = collections.deque()
        self.rejected: List[Request] = []
        self._batches = 0

    def _next_part(self, r: Request) -> Part:
        n = r.n - r.next_off if self.part_images == 0 else min(self.part_images, r.n - r.next_off)
        p = Part(r, r.next_off, n)
        r.next_off += n
        return p

    def arrive(self, r: Request) -> None:
        first = min(r.n, self.part_images) if self.part_images else r.n
        need = first * (r.L * r.L * 4 + POSE_BYTES)
        if need > self.hbm_budget:
            r.error = f"a part needs {need} bytes, more than the {self.hbm_budget}-byte device budget"
            self.rejected.append(r)
            return
        r.next_off = 0
        r.parts_left = 1 if self.part_images == 0 else -(-r.n // self.part_images)
        self.queue.append(self._next_part(r))

    def next_batch(self) -> Optional[Tuple[int, List[Part]]]:
        """Pop (slot, batch of parts) if the head part can be admitted now, else None."""
        if not self.queue or not self.free_slots:
            return None
        head = self.queue[0]
        if head.device_bytes > self.free_bytes:
            return None  # wait for memory: later parts do not overtake the head
        self.queue.popleft()
        batch = [head]
        used, imgs = head.device_bytes, head.n
        keep = collections.deque()
        while self.queue:
            p = self.queue.popleft()
            if (p.key == head.key and imgs + p.n <= self.max_batch_images
                    and used + p.device_bytes <= self.free_bytes):
                batch.append(p)
                used += p.device_bytes
                imgs += p.n
            else:
                keep.append(p)
        self.queue = keep
        self.free_bytes -= used
        slot = self.free_slots.pop(0)
        for p in batch:
            p.req.batch_id = self._batches
            if p.req.next_off < p.req.n:  # the request's next part
                if self.requeue == "back":
                    self.queue.append(self._next_part(p.req))
                else:
                    self.queue.appendleft(self._next_part(p.req))
        self._batches += 1
        return slot, batch

    def release(self, slot: int, batch: Sequence[Part]) -> None:
        self.free_bytes += sum(p.device_bytes for p in batch)
        self.free_slots.append(slot)
        self.free_slots.sort()


class Server:
    """Drives a :class:`Scheduler` and an executor over a stream of requests.

    The executor provides ``launch(slot, parts) -> token``, ``poll(token) ->
    bool`` and ``finish(token)`` (copies each part's results into its request).
    """

    def __init__(self, scheduler: Scheduler, executor, clock: Callable[[], float] = time.perf_counter,
                 idle_sleep: float = 50e-6, sleep: Callable[[float], None] = time.sleep):
        self.sched = scheduler
        self.exe = executor
        self.clock = clock
        self.idle_sleep = idle_sleep
        self.sleep = sleep

    def run(self, requests: Sequence[Request]) -> List[Request]:
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = self.clock()
        inflight: List[Tuple[object, int, List[Request]]] = []
        i = 0
        while i < len(pending) or inflight or self.sched.queue:
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                self.sched.arrive(pending[i])
                i += 1
            progressed = False
            still = []
            for tok, slot, batch in inflight:
                if self.exe.poll(tok):
                    try:
                        self.exe.finish(tok)
                    except Exception as e:  # a failed batch fails its requests, not the server
                        for p in batch:
                            p.req.error = f"{type(e).__name__}: {e}"
                    t = self.clock() - t0
                    for p in batch:
                        p.req.parts_left -= 1
                        if p.req.parts_left == 0:
                            p.req.done = t
                    self.sched.release(slot, batch)
                    progressed = True
                else:
                    still.append((tok, slot, batch))
            inflight = still
            while True:
                nb = self.sched.next_batch()
                if nb is None:
                    break
                slot, batch = nb
                t = self.clock() - t0
                for p in batch:
                    if math.isnan(p.req.admitted):
                        p.req.admitted = t
                try:
                    inflight.append((self.exe.launch(slot, batch), slot, batch))
                except Exception as e:
                    for p in batch:
                        p.req.error = f"{type(e).__name__}: {e}"
                        p.req.parts_left -= 1
                        if p.req.parts_left == 0:
                            p.req.done = self.clock() - t0
                    self.sched.release(slot, batch)
                progressed = True
            if not progressed:
                if not inflight and not self.sched.queue and i < len(pending):
                    wait = pending[i].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, 0.01))
                elif self.idle_sleep:
                    self.sleep(self.idle_sleep)
        return list(requests)


def summarize(requests: Sequence[Request]) -> dict:
    ok = [r for r in requests if not r.error]
    if not ok:
        return {"requests": 0, "rejected": len(requests)}
    lat = np.array([r.latency for r in ok]) * 1e3
    span = max(r.done for r in ok) - min(r.arrival for r in ok)
    imgs = sum(r.n for r in ok)
    return {
        "requests": len(ok), "rejected": len(requests) - len(ok), "images": imgs,
        "images_per_s": imgs / span if span > 0 else math.inf,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "span_s": span,
        "batches": len({r.batch_id for r in ok}),
    }


def serving_rings(L: int) -> Tuple[int, int]:
    """Rings 1..L/2-4 (keeps a 4-pixel margin for the shift grid at the box edge)."""
    return 1, L // 2 - 4


class GpuExecutor:
    """Runs batches through the library: one stream per slot, one handle per (slot, L)."""

    def __init__(self, ref_sets: Dict[Tuple[int, int], torch.Tensor], n_slots: int, precision: int,
                 shift_range: float = 3.0, shift_step: float = 1.0, mirror: int = 1, chunk_images: int = 2048,
                 device: int = 0):
        from . import Aligner
        self._Aligner = Aligner
        self.dev = torch.device("cuda", device)
        self.precision = precision
        self.geom = dict(shift_range=shift_range, shift_step=shift_step, mirror=mirror)
        self.chunk_images = chunk_images
        self.owners: Dict[Tuple[int, int], object] = {}
        st = torch.cuda.current_stream(self.dev)
        for (L, K), refs in ref_sets.items():
            a = self._aligner(L)
            a.set_refs(refs.to(self.dev, torch.float32).contiguous(), st)
            self.owners[(L, K)] = a
        torch.cuda.synchronize(self.dev)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_slots)]
        self.handles: List[Dict[int, object]] = [dict() for _ in range(n_slots)]
        self.loaded: List[Dict[int, int]] = [dict() for _ in range(n_slots)]
        self.launches = 0

    def _aligner(self, L: int):
        r1, r2 = serving_rings(L)
        return self._Aligner(L, r1, r2, 1, self.geom["shift_range"], self.geom["shift_step"], self.geom["mirror"],
                             self.precision, self.chunk_images)

    def launch(self, slot: int, batch: Sequence[Part]):
        from . import mra_align
        L, K = batch[0].key
        st = self.streams[slot]
        h = self.handles[slot].get(L)
        if h is None:
            h = self.handles[slot][L] = self._aligner(L)
        if self.loaded[slot].get(L) != K:
            h.copy_refs(self.owners[(L, K)], st)
            self.loaded[slot][L] = K
        n = sum(p.n for p in batch)
        with torch.cuda.stream(st):
            d_imgs = torch.empty((n, L, L), dtype=torch.float32, device=self.dev)
            d_poses = torch.empty((n, 8), dtype=torch.int32, device=self.dev)
            off = 0
            for p in batch:
                d_imgs[off:off + p.n].copy_(p.req.imgs[p.off:p.off + p.n], non_blocking=True)
                off += p.n
            mra_align(h.h, d_imgs, d_poses, st)
            h_poses = torch.empty((n, 8), dtype=torch.int32, pin_memory=True)
            h_poses.copy_(d_poses, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.launches += 1
        return {"ev": ev, "batch": list(batch), "bufs": (d_imgs, d_poses), "h_poses": h_poses, "slot": slot}

    def poll(self, tok) -> bool:
        return tok["ev"].query()

    def finish(self, tok) -> None:
        from . import mra_sync
        slot = tok["slot"]
        L = tok["batch"][0].key[0]
        mra_sync(self.handles[slot][L].h, self.streams[slot])  # surfaces a device wait timeout as an error
        off = 0
        for p in tok["batch"]:
            if p.req.poses is None:
                p.req.poses = torch.empty((p.req.n, 8), dtype=torch.int32)
            p.req.poses[p.off:p.off + p.n] = tok["h_poses"][off:off + p.n]
            off += p.n
        tok["bufs"] = None

    def close(self):
        for hs in self.handles:
            for a in hs.values():
                a.close()
        for a in self.owners.values():
            a.close()


# ---------------------------------------------------------------------------
# Synthetic request stream
# ---------------------------------------------------------------------------

BOX_SIZES = (64, 76, 96, 128)
REF_COUNTS = (50, 100, 200)


def draw_requests(n_requests: int, rate: float, seed: int, sizes=(200, 20000), boxes=BOX_SIZES,
                  ref_counts=REF_COUNTS) -> List[Request]:
    """Poisson arrivals at ``rate`` requests/s, sizes log-uniform on ``sizes``, (L, K) uniform."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests) if math.isfinite(rate) else np.zeros(n_requests)
    t = np.cumsum(gaps) - gaps[0]
    n = np.exp(rng.uniform(math.log(sizes[0]), math.log(sizes[1]), size=n_requests)).astype(np.int64)
    Ls = rng.choice(boxes, size=n_requests)
    Ks = rng.choice(ref_counts, size=n_requests)
    return [Request(i, int(Ls[i]), int(Ks[i]), int(n[i]), float(t[i])) for i in range(n_requests)]


def attach_stacks(requests: Sequence[Request], pools: Dict[int, torch.Tensor], seed: int) -> None:
    """Give each request a contiguous slice of the pinned particle pool for its box size."""
    rng = np.random.default_rng(seed)
    for r in requests:
        pool = pools[r.L]
        off = int(rng.integers(0, pool.shape[0] - r.n + 1))
        r.imgs = pool[off:off + r.n]


def make_pools(boxes, pool_images: int, n_classes: int, shift: int, snr: float, seed: int, device):
    """Particle pools per box size (pinned host) and the largest reference set per box (device).

    References follow the blob generator scaled to the box (20 Gaussians,
    sigma 3..8 px and disc radius 28 px at L = 76); particles are drawn from
    the first ``n_classes`` references so that every (L, K) set holds their
    true class.
    """
    import synth
    pools, refs = {}, {}
    for j, L in enumerate(boxes):
        s = L / 76.0
        R, blob = synth.make_refs(max(REF_COUNTS), L, blobs=20, sigma=(3.0 * s, 8.0 * s), disc=28.0 * s,
                                  seed=seed + 10 * j, device=device)
        refs[L] = R.float()
        truth = synth.draw_particle_truth(pool_images, n_classes, shift, True, seed + 10 * j + 1)
        imgs = synth.render_particles(blob, truth, snr=snr, noise_seed=seed + 10 * j + 2, device=device)
        host = torch.empty((pool_images, L, L), dtype=torch.float32, pin_memory=True)
        host.copy_(imgs.float())
        del imgs
        pools[L] = host
    return pools, refs


def run_stream(n_requests: int, loads: Sequence[float], precision: int, slots: int = 4,
               max_batch_images: int = 8192, hbm_budget: int = 32 << 30, calibration_requests: int = 40,
               pool_images: int = 20000, seed: int = 4004, device: int = 0, part_images: int = 0,
               requeue: str = "front") -> dict:
    """Calibrate capacity with a burst of requests, then serve Poisson streams at ``loads`` x capacity."""
    dev = torch.device("cuda", device)
    pools, refs = make_pools(BOX_SIZES, pool_images, 50, 3, 0.1, seed, dev)
    sets = {(L, K): refs[L][:K] for L in BOX_SIZES for K in REF_COUNTS}
    exe = GpuExecutor(sets, slots, precision, device=device)

    def serve(reqs):
        attach_stacks(reqs, pools, seed + 7)
        return summarize(Server(Scheduler(hbm_budget, slots, max_batch_images, part_images, requeue), exe).run(reqs))

    serve(draw_requests(min(8, calibration_requests), math.inf, seed + 2))  # first-use workspace allocation
    cal = serve(draw_requests(calibration_requests, math.inf, seed + 1))
    mean_n = (20000 - 200) / math.log(20000 / 200)  # mean of the log-uniform size law
    capacity = cal["images_per_s"] / mean_n
    report = {"workload": "Poisson stream; n log-uniform 200..20000; L in {64,76,96,128} (rings 1..L/2-4); "
                          "K in {50,100,200}; shifts +-3 step 1; mirror on",
              "slots": slots, "max_batch_images": max_batch_images, "part_images": part_images, "requeue": requeue,
              "hbm_budget_bytes": hbm_budget,
              "calibration": cal, "capacity_requests_per_s": capacity, "runs": {}}
    for load in loads:
        reqs = draw_requests(n_requests, load * capacity, seed + int(round(load * 1000)))
        report["runs"][f"{load:g}"] = dict(serve(reqs), offered_requests_per_s=load * capacity)
    report["gpu_launches"] = exe.launches
    exe.close()
    del pools
    return report


def _main():
    from . import MRA_BF16_RESCORE, MRA_FP16_RESCORE, MRA_FP32
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--load", type=float, nargs="+", default=[0.7, 0.5, 0.9])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-batch-images", type=int, default=8192)
    ap.add_argument("--hbm-budget-gb", type=float, default=32.0)
    ap.add_argument("--calibration-requests", type=int, default=40)
    ap.add_argument("--pool-images", type=int, default=20000)
    ap.add_argument("--part-images", type=int, default=0, help="0 serves each request as one part")
    ap.add_argument("--requeue", default="front", choices=["front", "back"])
    ap.add_argument("--seed", type=int, default=4004)
    args = ap.parse_args()
    prec = {"fp32": MRA_FP32, "bf16": MRA_BF16_RESCORE, "fp16": MRA_FP16_RESCORE}[args.precision]
    rep = run_stream(args.requests, args.load, prec, args.slots, args.max_batch_images,
                     int(args.hbm_budget_gb * 2**30), args.calibration_requests, args.pool_images, args.seed,
                     part_images=args.part_images, requeue=args.requeue)
    rep["precision"] = args.precision
    print(json.dumps(rep))


if __name__ == "__main__":
    _main()
