"""Host arithmetic of bench.py's roofline, on CPU: the tensor-core peaks per
arithmetic (BF16 hi+lo credits one product per three BF16 MMAs), no fixed
fallback for the FP32 / FP64 peaks (a fraction needs a measured peak), the
fraction itself, and the committed DRAM traffic applied only to its own
workload and kernel version."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _pk(**measured):
    pk = {"hbm_gbs": 6800.0, "bf16_tflops": 1935.7, "bf16_tflops_sustained": 1702.1,
          "source": "measured"}
    pk.update(measured)
    return pk


def test_tensor_peaks_per_arithmetic():
    pk = _pk(tf32_tflops=1056.0, fp32_tflops=69.8, fp64_tflops=1.1)
    assert bench.tensor_peak(pk, "bf16")[0] == 1935.7
    assert bench.tensor_peak(pk, "bf16x3")[0] == pytest.approx(1935.7 / 3)
    assert bench.tensor_peak(pk, "tf32")[0] == 1056.0
    assert bench.tensor_peak(pk, "fp32")[0] == 69.8
    assert bench.tensor_peak(pk, "fp64")[0] == 1.1
    # without this run's GEMM probes: TF32 from the BF16 peak and the nominal
    # ratio, FP32 / FP64 not at all
    bare = _pk()
    assert bench.tensor_peak(bare, "tf32")[0] == pytest.approx(1935.7 * 1.1 / 2.25)
    assert bench.tensor_peak(bare, "fp32")[0] is None
    assert bench.tensor_peak(bare, "fp64")[0] is None


def test_roofline_fraction_of_the_contraction():
    s = {"row": "a4", "launches": 2, "ms": 2 * 21.3, "bytes": 2 * 58.3e9, "flops": 2 * 8.55e12}
    r = bench.roofline_for("contract", s, _pk(), "bf16x3")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(8.55e12 / 21.3e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / (1935.7 / 3))
    hbm = bench.roofline_for("apply", {"row": "a1", "launches": 1, "ms": 19.5, "bytes": 87.7e9,
                                       "flops": 0.0}, _pk(), "bf16x3")
    assert hbm["bound"] == "hbm" and hbm["frac"] == pytest.approx(87.7e9 / 19.5e-3 / 1e9 / 6800.0)
    fp64 = bench.roofline_for("tridiag", {"row": "a6", "launches": 1, "ms": 7.2, "bytes": 0.0,
                                          "flops": 1.3e9}, _pk(), "bf16x3")
    assert fp64["peak"] is None and fp64["frac"] is None   # no measured FP64 peak: no fraction


def test_committed_traffic_only_for_its_workload_and_source():
    d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    e = d["contract"]
    got = bench.profiled_traffic("contract", e["workload"])
    import hashlib
    src = os.path.join(ROOT, "paper_1011_4764_gb300", "csrc", e["source"])
    current = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == e["source_sha"]
    assert got == (e["dram_bytes_per_launch"] if current else None)
    assert bench.profiled_traffic("contract", "some_other_workload") is None
    assert bench.profiled_traffic("no_such_kernel_class", e["workload"]) is None
