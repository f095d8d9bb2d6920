"""Host-side arithmetic of bench.py, on CPU: the rooflines' byte and gather counts, the clock record built from
nvidia-smi samples, and the rule that recorded ncu traffic is used only while the kernel's source is the one
it was taken on (every committed profile that carries a traffic figure must still match its kernel)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_of_one_iteration():
    # 1e6 x 5e5 with 2e7 nonzeros: two passes of 8 bytes per nonzero, u, ubar, v, vbar read and written.
    assert bench.algorithmic_bytes_per_iteration(10 ** 6, 5 * 10 ** 5, 2 * 10 ** 7) == 344_000_000
    assert bench.algorithmic_bytes_per_iteration(1, 1, 0) == 32


def test_gather_roofline_counts_one_gather_per_nonzero_per_pass():
    g = bench.gather_roofline(2 * 10 ** 7, 156e-6)
    assert g["gathers_per_launch"] == 4e7
    assert g["achieved_per_s"] == pytest.approx(4e7 / 156e-6)
    assert g["frac"] == pytest.approx(4e7 / 156e-6 / bench.GATHER_CEILING_PER_S)


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_takes_the_loaded_half_and_the_active_reasons():
    row = "0, {sm}, 2070, {w}, 0x0, Not Active, Not Active, Not Active, {cap}"
    lines = [row.format(sm=sm, w=300 + sm / 10, cap="Active" if sm == 1900 else "Not Active")
             for sm in (345, 345, 1900, 2070, 2070, 2070)]
    s = _sampler(lines + ["garbage", "0, [N/A], 2070"])
    assert s["sm_max_mhz"] == 2070.0 and s["samples"] == 6
    assert s["sm_mhz"] == 2070.0  # median of the upper half: idle samples before the load are left out
    assert s["reasons"] == ["sw_power_cap"]
    assert s["power_w_max"] == pytest.approx(507.0)
    thermal = _sampler(["0, 1500, 2070, 900, 0x0, Not Active, Active, Not Active, Not Active"])
    assert thermal["reasons"] == ["hw_thermal_slowdown"]
    assert _sampler([])["reasons"] == ["unsampled"]


def test_recorded_traffic_is_dropped_when_the_kernel_changed(tmp_path):
    f = tmp_path / "profile.txt"
    f.write_text("# a summary\nkernel = k\ntraffic_bytes_per_launch = 123456\nkernel_source_sha256 = abc\n")
    assert bench.recorded_traffic(str(f), lambda: "abc") == 123456.0
    assert bench.recorded_traffic(str(f), lambda: "abd") is None
    assert bench.recorded_traffic(str(tmp_path / "missing.txt"), lambda: "abc") is None


@pytest.mark.parametrize("path,source_hash", [
    (bench.TRAFFIC_FILE, bench.kernel_source_hash),
    (bench.BATCHED_TRAFFIC_FILE, bench.batched_source_hash),
    (bench.DENSE_TRAFFIC_FILE, bench.dense_source_hash),
    (bench.DENSE_F8_TRAFFIC_FILE, bench.dense_f8_source_hash),
])
def test_committed_profiles_match_their_kernels(path, source_hash):
    """A profile's DRAM traffic reaches the bench line only while its kernel is unchanged; a kernel edit
    without a new capture shows up here rather than as a silent null on the GPU machine."""
    t = bench.recorded_traffic(path, source_hash)
    assert t is not None and t > 0, os.path.basename(path)


def test_fp8_summary_arithmetic():
    N, k, T = 16384, 256, 300
    f8 = {"iter_s": 99e-6, "elapsed": 5 * 300 * 99e-6, "ub": np.zeros(4), "vb": np.ones(4),
          "spread_stored_matrix": 1.5, "spread_fp64_matrix": 1.5, "rms_stored_matrix": 0.1, "clocks": {}}
    bf = {"ub": np.zeros(4), "vb": np.ones(4)}
    peaks = {"bf16_tflops": 1900.0}
    s = bench.fp8_summary(N, k, T, 5, f8, bf, peaks, "measured")
    assert s["roofline"]["algorithmic_bytes_per_launch"] == 2 * N * N
    assert s["roofline"]["achieved"] == pytest.approx(2 * N * N / 99e-6 / 1e9)
    assert s["roofline"]["tensor"]["peak_tflops"] == 3800.0
    assert s["roofline"]["tensor"]["achieved_tflops"] == pytest.approx(4.0 * N * N * k / 99e-6 / 1e12)
    assert s["rel_diff_ubar_vbar_vs_bf16_run"] == 0.0
    assert s["probe_pairs_per_s"] == pytest.approx(k * T * 5 / f8["elapsed"])
