"""Host-side pieces of bench.py (no GPU): the algorithmic byte and flop models
of the roofline, the kernel each stage names, the end-to-end flush rule and
the rule that reports the committed ncu traffic figures."""
import json
import os

import numpy as np
import pytest

import bench

C2 = dict(n=1024, n_pad=2048, window=2056, records=1_200_000, kernel_width=7, tile=64)


def test_stage_bytes_of_the_benchmark_geometry():
    """The algorithmic model: grid values read and written once (8 B) and
    20 B per point (8 B value + 12 B record), whatever the plan's tables."""
    n, np_, W, m = 1024, 2048, 2056, 1 << 20
    for tables in (0, 1025 * 1026 * 8 + 1025 * 2048 * 8):
        b = bench.stage_bytes(dict(C2, phase_table_bytes=tables, points=m), m, 2, 8)
        assert b["col_fwd"] == 8 * (n * n + np_ * n)
        assert b["row_t2"] == 8 * (np_ * n + np_ * W)                 # 50.46 MB
        assert b["col_inv_fold"] == 8 * (np_ * W + W * W)
        assert b["interp"] == 8 * W * W + 20 * m
        b1 = bench.stage_bytes(dict(C2, phase_table_bytes=tables, points=m), m, 1, 8)
        assert b1["spread"] == 20 * m + 8 * W * W
        assert b1["row_t1"] == 8 * (np_ * W + np_ * n)
        assert b1["col_fwd_fold"] == 8 * (W * W + np_ * W)   # the window read once for both halves
        # summed over a solve: the survey's grid traffic 8(2P^2 + 2N'P + 2N'N + N^2) plus 20 B per point
        grid = 8 * (2 * W * W + 2 * np_ * W + 2 * np_ * n + n * n)
        assert sum(b1.values()) == grid + 20 * m
        assert sum(b.values()) == grid + 20 * m
    assert b["row_t2"] == 50_462_720


def test_plan_tables_are_reported_apart():
    m = 1 << 20
    equad = 1025 * 1026 * 8
    both = equad + 1025 * 2048 * 8
    t2 = bench.plan_table_bytes(dict(C2, phase_table_bytes=both, points=m), 2, 8)
    t1 = bench.plan_table_bytes(dict(C2, phase_table_bytes=both, points=m), 1, 8)
    assert t2["row_t2"] == 1025 * 2048 * 8        # the Tx-folded rows
    assert t1["row_t1"] == equad                   # the E quadrant
    only_e = bench.plan_table_bytes(dict(C2, phase_table_bytes=equad, points=m), 2, 8)
    assert only_e["row_t2"] == equad
    assert t2["interp"] == 4 * m                   # 16-byte records against the 12-byte model
    assert t1["spread"] == 16 * C2["records"] - 12 * m + 8 * (C2["records"] - m)


def test_stage_flops_model():
    f = bench.stage_flops(C2, 1 << 20, 2)
    fft = 5.0 * 2048 * np.log2(2048)
    assert f["col_fwd"] == pytest.approx(1024 * fft)
    assert f["row_t2"] == pytest.approx(3 * 2048 * fft + 6.0 * 2048 * 2048)
    w = 7
    assert f["interp"] == pytest.approx((4 * w * (w + 1) + 4 * w * w + 4 * w) * (1 << 20))
    f64 = bench.stage_flops(dict(C2, kernel_width=13), 1000, 2, True)
    assert f64["interp"] == pytest.approx((4 * 13 * 13 + 4 * 13 * 13 + 4 * 13) * 1000)


@pytest.mark.parametrize("tile,f64,w,want", [
    (64, False, 7, "spread_fixed_kernel<7, true, 2>"),
    (32, False, 7, "spread_private_kernel<float, 7, true>"),
    (64, False, 13, "spread_fixed_kernel<16, false, 2>"),
    (16, True, 13, "spread_private_kernel<double, 13, true>"),
    (64, True, 13, "spread_kernel<double, 13, true>"),
    (64, True, 11, "spread_kernel<double, 11, true>"),
])
def test_spreading_kernel_names(tile, f64, w, want):
    assert bench.kernel_of_stage("spread", dict(n_pad=2048, kernel_width=w, tile=tile), f64) == want


@pytest.mark.parametrize("split,want", [(0, "spread_df_kernel<13>"), (40, "spread_df_kernel<13>")])
def test_double_float_kernel_names(split, want):
    """FP64 plans on the double-float path name the double-float kernels, and
    their gridding stages take the double-float roof (FP32 lane rate / 12
    instructions per 2-flop multiply-add)."""
    info = dict(n_pad=2048, kernel_width=13, tile=16, double_float=1, spread_split_ctas=split)
    assert bench.kernel_of_stage("spread", info, True) == want
    assert bench.kernel_of_stage("interp", info, True) == "interp_df_kernel<13>"
    assert bench.DF_PEAK_TFLOPS == pytest.approx(152 * 128 * 2.07e9 / 6 / 1e12)


def test_fp64_row_pass_names_follow_the_size_rule():
    """FP64 row (and column) passes run in double-float from N' = 512 up, in FP64 below."""
    assert bench.kernel_of_stage("row_t1", dict(n_pad=4096, kernel_width=13), True) == "row_t1_kernel<dfc, 12>"
    assert bench.kernel_of_stage("row_t2", dict(n_pad=512, kernel_width=13), True) == "row_t2_kernel<dfc, 9>"
    assert bench.kernel_of_stage("row_t1", dict(n_pad=128, kernel_width=13), True) == "row_t1_kernel<double2, 7>"
    assert bench.kernel_of_stage("row_t2", dict(n_pad=2048, kernel_width=7), False) == "row_t2_kernel<float2, 11>"


def test_column_kernel_names_follow_the_tma_rule():
    assert bench.kernel_of_stage("col_inv_fold", dict(n_pad=2048, kernel_width=7), False) == "col_tma_kernel<11, 3>"
    assert bench.kernel_of_stage("col_fwd", dict(n_pad=2048, kernel_width=7), False) == "col_kernel<float2, 11, 2>"
    assert bench.kernel_of_stage("col_fwd", dict(n_pad=4096, kernel_width=7), False) == "col_tma_kernel<12, 2>"
    assert bench.kernel_of_stage("col_inv_fold", dict(n_pad=2048, kernel_width=13), True) == \
        "col_kernel<dfc, 11, 3>"
    assert bench.kernel_of_stage("col_fwd_fold", dict(n_pad=128, kernel_width=13), True) == \
        "col_kernel<double2, 7, 0>"


def test_e2e_flush_rule():
    assert bench.e2e_needs_flush(0.8e6)            # a 64^2 plane stays in L2
    assert not bench.e2e_needs_flush(211e6)        # the benchmark plane does not
    assert bench.e2e_needs_flush(211e6, lanes=2)   # one other lane: 211 MB < 2 x 129 MB


def test_traffic_is_reported_only_for_the_profiled_source(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    rec = t["row_t2"]
    monkeypatch.setattr(bench, "source_hash", lambda stage: rec["source_hash"])
    assert bench.measured_traffic("row_t2") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "source_hash", lambda stage: "0" * 16)
    assert bench.measured_traffic("row_t2") is None
    assert bench.measured_traffic("no_such_stage") is None
