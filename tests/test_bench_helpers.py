"""Host-side arithmetic of bench.py's JSON line: the roofline of the main
BaseCase launch and the DRAM traffic scaled from the recorded capture."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_scales_the_capture_per_point_pair():
    b, p = bench.TRAFFIC_CAPTURE[("powerlaw64", "bf16")]
    assert bench.traffic_of("powerlaw64", "bf16", p) == pytest.approx(b)
    assert bench.traffic_of("powerlaw64", "bf16", 2 * p) == pytest.approx(2 * b)
    # about 1.8 bytes of DRAM per point pair at d = 64 (288-byte operand
    # rows shared by a 128-query chunk are 2.25 B per pair)
    assert 1.0 < b / p < 2.25


def test_no_capture_means_no_traffic():
    assert bench.traffic_of("gmm16", "bf16", 1e12) is None
    assert bench.traffic_of("powerlaw64", "fp32", 1e12) is None


def test_tensor_roofline_counts_two_flops_per_coordinate():
    r = bench.roofline("bf16", 64, pairs=1e12, ns_tile=1e9, sms=152, traffic=None)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["algorithmic_flops_per_step"] == pytest.approx(2 * 64 * 1e12)
    assert r["achieved"] == pytest.approx(128.0)   # 1.28e14 flops in one second
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    t = bench.roofline("tf32", 64, pairs=1e12, ns_tile=1e9, sms=152, traffic=None)
    assert t["peak"] == pytest.approx(r["peak"] * 1.1 / 2.25)


def test_cuda_core_roofline_is_the_alu_peak():
    r = bench.roofline("fp32", 16, pairs=1e12, ns_tile=2e9, sms=152, traffic=None)
    assert r["bound"] == "alu"
    assert r["algorithmic_flops_per_step"] == pytest.approx(3 * 16 * 1e12)
    assert r["achieved"] == pytest.approx(24.0)
    # 2 flops x 128 lanes x 152 SMs at the SM clock (2070 MHz unless measured otherwise)
    assert 70.0 < r["peak"] < 90.0
