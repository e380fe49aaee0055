"""Host logic of bench.py's roofline objects: the algorithmic work per launch
of each kernel family, and the per-kernel table agreeing with the top-level
object for the same kernel (one source of work counts)."""
import importlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_work_counts_per_launch(bench):
    px = bench.H * bench.W * 2
    # tensor-core hidden conv: 32 BF16 channels in and out per pixel
    assert bench.algorithmic("conv3x3_tc_bf16", 8, 2)[:3] == ("hbm", "GB/s", 128.0 * px)
    # flexible network: the step's pointwise multiply-adds spread over its launches
    from paper_2403_03488_gb300.flnet import work_per_pixel
    b, u, w, _, _ = bench.algorithmic("fl_pw_fwd", 15, 2)
    assert (b, u) == ("alu", "TFLOP/s") and w == pytest.approx(2 * work_per_pixel()["pw_macs"] * px / 15)
    b, u, w, _, _ = bench.algorithmic("fl_dw3x3_fwd", 14, 2)
    assert (b, u) == ("hbm", "GB/s") and w == pytest.approx(work_per_pixel()["dw_bytes"] * px / 14)
    # matcher: 192 FLOP per (reference, candidate) pair, two launches (passes) per step
    b, u, w, _, _ = bench.algorithmic("bm3d_match_fp32", 2, 2)
    assert w == 192.0 * bench.match_pairs(bench.H, bench.W) * 2


def test_table_matches_top_level_object(bench):
    res = {"conv3x3_tc_bf16": (8, 1.0), "fl_pw_fwd": (15, 10.0), "nlm_fp32": (1, 0.9),
           "bm3d_match_fp32": (2, 24.0), "pack_w_tc": (8, 0.05)}
    table = bench.kernel_rooflines(res, 1, 2)
    assert "pack_w_tc" not in table  # no plain work count: not reported
    for k, (n, ms) in res.items():
        if k not in table:
            continue
        bound, unit, work, peak, _ = bench.algorithmic(k, n, 2)
        ach = work / (ms / n / 1e3) / (1e12 if unit == "TFLOP/s" else 1e9)
        assert table[k]["bound"] == bound and table[k]["unit"] == unit
        assert table[k]["achieved"] == pytest.approx(ach, rel=1e-3)
        assert table[k]["frac"] == pytest.approx(ach / peak, abs=1e-4)


def test_filter_counts_per_pixel(bench):
    """The dense-contraction counts of the two filtering passes per pixel of a
    1024 x 1024 image (full groups): 36 kFLOP (pass 1: 2D DCT forward and back
    as 64 x 64 products, 16 x 16 Walsh-Hadamard both ways) and 130 kFLOP
    (pass 2: three of each with 32-patch groups)."""
    px = 1024 * 1024
    t1, a1 = bench.filter_work(False, 1024, 1024, 1)
    t2, a2 = bench.filter_work(True, 1024, 1024, 1)
    assert t1 / px == pytest.approx(36.1e3, rel=0.01)
    assert t2 / px == pytest.approx(130.0e3, rel=0.01)
    # the separable form does about a quarter of the 2D-transform work
    assert 0.15 < a1 / t1 < 0.4 and 0.15 < a2 / t2 < 0.4


def test_fp32_peak_from_device_numbers(bench):
    hw = {"sm_count": 152, "sm_mhz": 2070.0, "source": "test"}
    assert bench.fp32_peak(hw) == pytest.approx(80.56, rel=1e-3)
    hw2 = dict(hw, sm_count=144, sm_mhz=1900.0)
    b, u, w, peak, note = bench.algorithmic("bm3d_match_fp32", 2, 2, hw2)
    assert peak == pytest.approx(144 * 128 * 2 * 1.9e9 / 1e12) and "144 SM" in note


def test_larger_patch_work_counts():
    """The larger-patch counts reduce to the 8 x 8 ones at k = 8 (2048 FLOP per
    separable 2D DCT, 8192 per dense one) and scale with k as the definitions
    say: 4 k^3 per separable 2D DCT, 2 k^4 per dense one, 3 k^2 per matching pair."""
    import bench
    t8, a8 = bench.filter_flops_per_patch(False, 16, 8)
    assert t8 == 2 * 2 * 64 * 64 + 2 * 2 * 16 * 64
    assert a8 == 2 * 2048 + 2 * 64 * 4 + 2 * 64 + 3 * 64
    t12, a12 = bench.filter_flops_per_patch(True, 32, 12)
    assert t12 == 3 * 2 * 144 * 144 + 3 * 2 * 32 * 144
    assert a12 == 3 * 4 * 12 ** 3 + 3 * 144 * 5 + 4 * 144 + 3 * 144
    assert bench.match_pairs(40, 40, 3, 39, 8) == bench.match_pairs(40, 40)
    old = (bench.H, bench.W)
    try:
        bench.H = bench.W = 64
        b, u, w, _, _ = bench.algorithmic("bm3d_match_pre_large", 1, 2)
        assert (b, u) == ("alu", "TFLOP/s") and w == 3.0 * 144 * bench.match_pairs(64, 64, 4, 39, 12) * 2
    finally:
        bench.H, bench.W = old
