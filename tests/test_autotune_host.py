"""Host logic of the launch autotuner (no GPU): which candidates a configuration gets."""
from paper_2011_05755_gb300 import (MRA_BF16_RESCORE, MRA_FP16_RESCORE, MRA_FP32, MRA_KERNEL_AUTO,
                                    MRA_KERNEL_MMA_SYNC, MRA_KERNEL_TCGEN05)
from paper_2011_05755_gb300.autotune import _ring_M, candidates


def test_ring_length_of_the_largest_ring():
    assert _ring_M(1, 35, 1) == 256      # 2 pi 35 = 220 -> 256
    assert _ring_M(1, 60, 1) == 512
    assert _ring_M(3, 25, 3) == 256      # rings 3, 6, ..., 24: the largest is 24
    assert _ring_M(1, 12, 1) == 128


def test_kernel_variants_only_where_two_exist():
    for prec in (MRA_BF16_RESCORE, MRA_FP16_RESCORE):
        ks = {k for k, _ in candidates(1, 35, 1, prec)}
        assert ks == {MRA_KERNEL_MMA_SYNC, MRA_KERNEL_TCGEN05}
        assert {k for k, _ in candidates(1, 60, 1, prec)} == {MRA_KERNEL_AUTO}   # M = 512: one kernel
    assert {k for k, _ in candidates(1, 35, 1, MRA_FP32)} == {MRA_KERNEL_AUTO}
    assert all(c >= 0 for _, c in candidates(1, 35, 1, MRA_BF16_RESCORE))
