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
