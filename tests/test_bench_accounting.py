"""The bench's algorithmic-work accounting (the numerators of its rooflines)
and the DRAM-traffic table it reads, checked on the CPU.

The per-pair flop counts are the closed forms of the method's two steps:
the contraction costs 8 real flops per (ring, frequency) bin with
N_r / 2 >= f (four real products and their sums, Sec. 2's integrand in
Fourier space), the inverse angular FFT 5 M log2 M; the polar stage
2.5 N log2 N + 9 N per ring (real FFT plus a 9-flop bilinear sample).
"""
import json
import math
import os

import pytest

import bench
from oracle import mra_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("r1,r2,dr", [(1, 35, 1), (1, 60, 1), (2, 20, 2), (5, 12, 1)])
def test_bench_ring_table_matches_the_oracle(r1, r2, dr):
    assert bench.ring_table(r1, r2, dr) == [tuple(x) for x in O.ring_table(r1, r2, dr)]


def test_per_pair_work_of_the_two_workloads():
    # rings 1..35 (M = 256): R_f = 35, 34, 33, 30, 25, 15 by f-range -> sum_f R_f = 2815
    assert bench.path_work(256, bench.ring_table(1, 35, 1)) == (8 * 2815, 5 * 256 * 8)
    # rings 1..60 (M = 512): sum_f R_f = 8600
    assert bench.path_work(512, bench.ring_table(1, 60, 1)) == (8 * 8600, 5 * 512 * 9)
    # sum_f R_f is the number of complex bins sum_r (N_r / 2 + 1)
    for rings in (bench.ring_table(1, 35, 1), bench.ring_table(1, 60, 1), bench.ring_table(3, 17, 2)):
        M = max(n for _, n in rings)
        assert bench.path_work(M, rings)[0] == 8 * sum(n // 2 + 1 for _, n in rings)


def test_polar_row_work():
    rings = bench.ring_table(1, 35, 1)
    assert sum(n for _, n in rings) == 5560
    assert sum(2.5 * n * math.log2(n) + 9.0 * n for _, n in rings) == pytest.approx(155460.0)


def test_traffic_table_entries_are_complete():
    table = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert {"cc_tc256_kernel", "polar_fft_kernel", "cc_fp32_kernel"} <= set(table)
    for name, ent in table.items():
        assert os.path.isfile(os.path.join(ROOT, ent["capture"])), name
        for src in ent["sources"]:
            assert os.path.isfile(os.path.join(ROOT, src)), (name, src)
        assert len(ent["source_hash"]) == 16 and ent["bytes_per_unit"] > 0, name


def test_traffic_is_close_to_the_algorithmic_bytes():
    """Measured DRAM bytes per unit against the data each kernel must move:
    the 16-bit particle fragments (KS k-steps x 64 B per row) once, plus 8 B
    of row maxima per pair (contraction), or written once (polar).  Writes
    still in L2 when a launch ends are not counted, hence the lower margin."""
    table = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))

    def ks(rings):
        M = max(n for _, n in rings)
        return sum(-(-sum(1 for _, n in rings if n // 2 >= f) // 16) for f in range(M // 2 + 1))

    ks76, ks128 = ks(bench.ring_table(1, 35, 1)), ks(bench.ring_table(1, 60, 1))
    assert (ks76, ks128) == (211, 708)
    tc256 = ks76 * 64 / 100 + 8          # K = 100
    tc512 = ks128 * 64 / 200 + 8         # K = 200
    polar = ks76 * 64
    assert 0.97 * tc256 <= table["cc_tc256_kernel"]["bytes_per_unit"] <= 1.2 * tc256
    assert 0.97 * tc512 <= table["cc_tc512_kernel"]["bytes_per_unit"] <= 1.2 * tc512
    assert 0.95 * polar <= table["polar_fft_kernel"]["bytes_per_unit"] <= 1.2 * polar
    # tcgen05 path: frequencies four to an MMA in f order, a group's k-steps those of its lowest
    # frequency; 4 KB of particle operand per 16 rows and k-step
    rings = bench.ring_table(1, 35, 1)
    nu = sum(-(-sum(1 for _, n in rings if n // 2 >= f) // 16) for f in range(0, 129, 4))
    assert nu == 55
    umma = nu * 4096 / 16 / 100 + 8
    assert 0.97 * umma <= table["cc_umma256_kernel"]["bytes_per_unit"] <= 1.2 * umma
