"""Host-side logic of bench.py's roofline entries (no GPU).

The Gram kernel's algorithmic work per launch is n * 2w * 2d flops (each
point against its 2w window neighbours) and, per point, the operand row (2
ceil64(d) BF16 or ceil128(d) FP8 bytes), the point's list read and written
(2 KP x 8 bytes, KP = 16/32 >= k + slack) and its (norm, scale) and id (12
bytes); the plain window kernel's work is 3 flops per (pair, coordinate)
over the n w - w(w+1)/2 pairs of one tree. The DRAM
traffic figure is only reported while the kernel's source file is the one the
counters were taken on.
"""
import hashlib
import os

import pytest

import bench


class _A:
    n, d, k, w, tensor_slack, mode = 3_000_000, 384, 15, 32, -1, "tensor"


def test_gram_work_full_size():
    flops, per_point = bench.gram_work(_A)
    assert per_point == 2 * 384 + 2 * 16 * 8 + 12 == 1036
    assert flops == 2.0 * 3_000_000 * 2 * 32 * 384


def test_gram_roofline_narrow_window_is_hbm_side():
    """At w = 32 the band's flops are few: the bytes decide the bound."""
    r = bench.gram_roofline(_A, launch_ms=1.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1036 * 3_000_000 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_gram_roofline_wide_window_is_tensor_bound():
    class A(_A):
        w = 512
    r = bench.gram_roofline(A, launch_ms=2.0, gather_ms=0.7)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    flops = 2.0 * 3_000_000 * 1024 * 384
    assert r["achieved"] == pytest.approx(flops / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["gather"]["bytes"] == 2.0 * 3_000_000 * 768 + 16.0 * 3_000_000


@pytest.mark.parametrize("d,k,slack,per_point", [(16, 10, -1, 2 * 64 + 2 * 16 * 8 + 12),   # d padded to 64, KP 16
                                                 (100, 15, -1, 2 * 128 + 2 * 16 * 8 + 12),  # KP 16 holds k + 1 = 16
                                                 (384, 16, -1, 2 * 384 + 2 * 32 * 8 + 12),  # k + 1 = 17 needs KP 32
                                                 (384, 15, 17, 2 * 384 + 2 * 32 * 8 + 12)])  # k + slack = 32
def test_gram_bytes_per_point_rounding(d, k, slack, per_point):
    class A(_A):
        pass
    A.d, A.k, A.tensor_slack = d, k, slack
    assert bench.gram_work(A)[1] == per_point


def test_fp8_rows_and_peak():
    class A(_A):
        mode, w, tensor_slack = "fp8", 512, 17
    flops, per_point = bench.gram_work(A, fp8=True)
    assert per_point == 384 + 2 * 32 * 8 + 12
    r = bench.gram_roofline(A, launch_ms=1.0)
    peaks, _ = bench.measured_peaks()
    base = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    assert r["peak"] == pytest.approx(2 * base)


def test_window_flops():
    r = bench.window_roofline(_A, launch_ms=1.0)
    pairs = 3_000_000 * 32 - 32 * 33 // 2
    assert r["achieved"] == pytest.approx(3.0 * 384 * pairs / 1e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2070e6 * 1.5 / 1e12)


def test_traffic_only_for_the_captured_source():
    src = open(os.path.join(bench.ROOT, "paper_2508_21682_gb300", "csrc", "gram.cu"), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    assert bench.traffic_per_launch({"bytes_per_point": 1000, "source_sha": sha, "file": "gram.cu"}, 10) == 10000
    assert bench.traffic_per_launch({"bytes_per_point": 1000, "source_sha": "0" * 16, "file": "gram.cu"}, 10) is None
    assert bench.traffic_per_launch({"bytes_per_point": None, "source_sha": sha, "file": "gram.cu"}, 10) is None


def test_measured_peaks_or_fallback():
    peaks, src = bench.measured_peaks()
    assert src in ("of measured", "of fallback")
    assert float(peaks["hbm_gbs"]) > 0


def test_cpp_oracle_baseline_on_a_tiny_sample():
    """The C++ oracle's share of the CPU baseline: threads x sample points per
    second of wall time, scaled from the sample's trees to the workload's."""
    class A:
        n, d, T, w, k, nq, search_w, components, bits = 100_000, 8, 16, 4, 5, 1000, 4, 5, 8

    val, wall = bench.cpp_oracle_parallel(A, 2, 200, 1)
    assert wall > 0
    assert val == pytest.approx(2 * 200 / (wall * 16))
