"""Serving loop: scheduling policy on the host (fake executor, simulated
clock) and, on the GPU, that every request's poses are the same served
alone, in a concurrent mix, and through a plain mra_align call."""
import math

import numpy as np
import pytest
import torch

from paper_2011_05755_gb300.serve import (Request, Scheduler, Server, draw_requests, serving_rings,
                                          summarize)


class SimClock:
    def __init__(self, dt=1e-3):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t

    def sleep(self, s):
        self.t += s


class FakeExecutor:
    """Batch of n images takes n * per_image seconds of simulated time."""

    def __init__(self, clock, per_image=1e-4, fail_key=None):
        self.clock = clock
        self.per_image = per_image
        self.fail_key = fail_key
        self.log = []
        self.in_use = 0
        self.max_in_use = 0

    def launch(self, slot, batch):
        if batch[0].key == self.fail_key:
            raise RuntimeError("injected launch failure")
        n = sum(p.n for p in batch)
        self.in_use += sum(p.device_bytes for p in batch)
        self.max_in_use = max(self.max_in_use, self.in_use)
        tok = {"end": self.clock.t + n * self.per_image, "batch": batch, "slot": slot}
        self.log.append(("launch", self.clock.t, slot, [p.req.rid for p in batch]))
        return tok

    def poll(self, tok):
        return self.clock.t >= tok["end"]

    def finish(self, tok):
        self.in_use -= sum(p.device_bytes for p in tok["batch"])
        for p in tok["batch"]:
            if p.req.poses is None:
                p.req.poses = np.full((p.req.n, 8), -1)
            p.req.poses[p.off:p.off + p.n] = p.req.rid
        self.log.append(("finish", self.clock.t, tok["slot"], [p.req.rid for p in tok["batch"]]))


def _run(reqs, budget, slots, max_batch, per_image=1e-4, fail_key=None, part_images=0, requeue="front"):
    clk = SimClock()
    exe = FakeExecutor(clk, per_image, fail_key)
    srv = Server(Scheduler(budget, slots, max_batch, part_images, requeue), exe, clock=clk, idle_sleep=1e-4,
                 sleep=clk.sleep)
    srv.run(reqs)
    return exe


def test_draw_requests_is_seeded_and_in_range():
    a = draw_requests(500, 10.0, seed=3)
    b = draw_requests(500, 10.0, seed=3)
    assert [(r.n, r.L, r.K, r.arrival) for r in a] == [(r.n, r.L, r.K, r.arrival) for r in b]
    n = np.array([r.n for r in a])
    assert n.min() >= 200 and n.max() < 20000
    # log-uniform: the median is near the geometric mean sqrt(200 * 20000) = 2000
    assert 1400 < np.median(n) < 2800
    gaps = np.diff([r.arrival for r in a])
    assert (gaps >= 0).all() and 0.07 < gaps.mean() < 0.13   # Poisson at 10/s
    assert {r.L for r in a} == {64, 76, 96, 128} and {r.K for r in a} == {50, 100, 200}
    assert serving_rings(76) == (1, 34) and serving_rings(128) == (1, 60)


def test_every_request_completes_within_the_memory_budget():
    reqs = draw_requests(120, 200.0, seed=5, sizes=(20, 400), boxes=(32, 48), ref_counts=(4, 8))
    budget = 4 * 400 * 48 * 48 * 4
    exe = _run(reqs, budget, slots=3, max_batch=600)
    assert all(not r.error and r.poses is not None for r in reqs)
    assert all(r.done >= r.admitted >= r.arrival for r in reqs)
    assert exe.max_in_use <= budget
    s = summarize(reqs)
    assert s["requests"] == 120 and s["p99_ms"] >= s["p50_ms"] > 0


def test_batching_merges_only_same_key_up_to_the_image_cap():
    reqs = [Request(0, 32, 4, 100, 0.0), Request(1, 32, 4, 100, 0.0), Request(2, 48, 4, 100, 0.0),
            Request(3, 32, 4, 300, 0.0), Request(4, 32, 4, 250, 0.0)]
    exe = _run(reqs, 10**9, slots=1, max_batch=450)
    launches = [e[3] for e in exe.log if e[0] == "launch"]
    assert launches[0] == [0, 1, 4]       # 100 + 100 + 250 <= 450; 300 would exceed it
    assert sorted(sum(launches, [])) == [0, 1, 2, 3, 4]
    for b in launches:
        assert len({reqs[i].key for i in b}) == 1


def test_slot_is_refilled_while_others_still_run():
    # one long and two short requests on two slots, then a queued one:
    # it must start when the first short batch ends, not after the long one
    reqs = [Request(0, 32, 4, 5000, 0.0), Request(1, 48, 4, 100, 0.0), Request(2, 48, 8, 100, 0.0)]
    exe = _run(reqs, 10**9, slots=2, max_batch=10**6)
    fin1 = next(e[1] for e in exe.log if e[0] == "finish" and e[3] == [1])
    start2 = next(e[1] for e in exe.log if e[0] == "launch" and e[3] == [2])
    fin0 = next(e[1] for e in exe.log if e[0] == "finish" and e[3] == [0])
    assert fin1 <= start2 < fin0


def test_head_is_not_overtaken_and_oversized_is_rejected():
    big = Request(1, 48, 4, 1000, 0.0)
    reqs = [Request(0, 48, 4, 1000, 0.0), big, Request(2, 32, 4, 10, 0.001), Request(3, 48, 4, 10**7, 0.0)]
    budget = 1000 * (48 * 48 * 4 + 32) + 10 * (32 * 32 * 4 + 32)
    exe = _run(reqs, budget, slots=4, max_batch=1)
    assert reqs[3].error and "budget" in reqs[3].error
    order = [e[3][0] for e in exe.log if e[0] == "launch"]
    assert order.index(1) < order.index(2)    # FIFO: the small request waits behind the head


def test_parts_round_robin_interleaves_small_requests():
    # a large request first, then small ones arriving just after it, one slot
    reqs = [Request(0, 32, 4, 1000, 0.0)] + [Request(i, 48, 4, 50, 0.001 * i) for i in range(1, 4)]
    exe = _run(reqs, 10**9, slots=1, max_batch=10**6, part_images=300, requeue="back")
    for r in reqs:
        assert not r.error and (r.poses == r.rid).all()   # every image served exactly by its own request
    # served whole, request 0 would finish before the small ones start; in parts they finish first
    assert all(reqs[i].done < reqs[0].done for i in (1, 2, 3))
    launched = [e[3] for e in exe.log if e[0] == "launch"]
    assert sum(1 for b in launched if 0 in b) == 4       # ceil(1000 / 300) parts
    fifo = [Request(0, 32, 4, 1000, 0.0)] + [Request(i, 48, 4, 50, 0.001 * i) for i in range(1, 4)]
    _run(fifo, 10**9, slots=1, max_batch=10**6, part_images=0)
    assert all(fifo[i].done > fifo[0].done for i in (1, 2, 3))


def test_parts_front_spread_a_large_request_over_the_slots():
    whole = [Request(0, 32, 4, 1200, 0.0)]
    _run(whole, 10**9, slots=4, max_batch=10**6, part_images=0)
    split = [Request(0, 32, 4, 1200, 0.0)]
    exe = _run(split, 10**9, slots=4, max_batch=300, part_images=300, requeue="front")
    assert (split[0].poses == 0).all()
    slots = {e[2] for e in exe.log if e[0] == "launch"}
    assert len(slots) == 4                                   # the four parts ran side by side
    assert split[0].done < 0.5 * whole[0].done


def test_failed_batch_fails_only_its_requests():
    reqs = [Request(0, 32, 4, 50, 0.0), Request(1, 48, 8, 50, 0.0), Request(2, 32, 4, 50, 0.0)]
    _run(reqs, 10**9, slots=2, max_batch=10**6, fail_key=(48, 8))
    assert reqs[1].error.startswith("RuntimeError")
    assert not reqs[0].error and not reqs[2].error


# ---------------------------------------------------------------------------
# GPU: alone == mix == plain mra_align
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mra():
    import __graft_entry__ as entry
    entry.build()
    import paper_2011_05755_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    return m


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_results_same_alone_and_in_the_mix(mra, prec):
    from paper_2011_05755_gb300.serve import GpuExecutor, attach_stacks, make_pools
    precision = mra.MRA_FP32 if prec == "fp32" else mra.MRA_BF16_RESCORE
    dev = torch.device("cuda", 0)
    boxes, counts = (32, 48), (4, 6)
    pools, refs = make_pools(boxes, 1200, 4, 3, 0.5, 77, dev)
    sets = {(L, K): refs[L][:K] for L in boxes for K in counts}

    def fresh():
        return draw_requests(14, math.inf, seed=9, sizes=(20, 400), boxes=boxes, ref_counts=counts)

    exe = GpuExecutor(sets, 3, precision, chunk_images=256)
    mix = fresh()
    attach_stacks(mix, pools, 5)
    Server(Scheduler(2**30, 3, 700, part_images=90), exe).run(mix)
    assert all(not r.error for r in mix)
    assert len({r.batch_id for r in mix}) < len(mix)          # something was batched
    for r in mix:
        alone = fresh()[r.rid]
        alone.imgs = r.imgs
        Server(Scheduler(2**30, 1, 1), exe).run([alone])
        assert not alone.error, (r.rid, alone.error)
        assert torch.equal(alone.poses, r.poses), r.rid
        r1, r2 = serving_rings(r.L)
        a = mra.Aligner(r.L, r1, r2, 1, 3.0, 1.0, 1, precision)
        a.set_refs(sets[r.key].to(dev).contiguous())
        direct = a.align(r.imgs.to(dev)).cpu()
        a.close()
        assert torch.equal(direct, r.poses), r.rid
    exe.close()
