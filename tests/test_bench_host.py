"""Host-side logic of bench.py's roofline entries (no GPU).

The Gram kernel's algorithmic bytes per point are the BF16 row (2 ceil64(d)),
the point's list read and written (2 KP x 8 bytes, KP = 16/32/64 >= k + 1) and
its id and norm (8 bytes); the plain window kernel's work is 3 flops per
(pair, coordinate) over the n w - w(w+1)/2 pairs of one tree. The DRAM
traffic figure is only reported while the kernel's source file is the one the
counters were taken on.
"""
import hashlib
import os

import pytest

import bench


class _A:
    n, d, k, w = 3_000_000, 384, 15, 32


def test_gram_bytes_per_point_full_size():
    r = bench.gram_roofline(_A, launch_ms=1.0)
    assert r["bytes_per_point"] == 2 * 384 + 2 * 16 * 8 + 8 == 1032
    assert r["bytes_per_launch"] == 1032 * 3_000_000
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1032 * 3_000_000 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


@pytest.mark.parametrize("d,k,per_point", [(16, 10, 2 * 64 + 2 * 16 * 8 + 8),   # d padded to 64, KP 16
                                           (100, 15, 2 * 128 + 2 * 16 * 8 + 8),  # KP 16 holds k + 1 = 16
                                           (384, 16, 2 * 384 + 2 * 32 * 8 + 8),  # k + 1 = 17 needs KP 32
                                           (384, 40, 2 * 384 + 2 * 64 * 8 + 8)])
def test_gram_bytes_per_point_rounding(d, k, per_point):
    class A(_A):
        pass
    A.d, A.k = d, k
    assert bench.gram_roofline(A, 1.0)["bytes_per_point"] == per_point


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
