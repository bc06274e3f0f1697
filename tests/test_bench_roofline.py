"""The bench line's roofline arithmetic (host logic, CPU): achieved flops from the scope table's
per-cell count, the derived FMA peaks from unit counts and clocks, the peak scaled from the measured
bf16 rate, the algorithmic-bytes fraction of HBM, the traffic record's source check, and the order
of the roofline object (the kernel with the largest launch-list share leads)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CELLS, DOFS = 32 ** 3, 859812


def test_derived_fma_peaks():
    # 152 SMs x 128 FP32 lanes (2 FP64 lanes) x 2 flops x 2.07 GHz
    assert bench.alu_peak_tflops(32, 152, 2070.0) == pytest.approx(80.548, rel=1e-4)
    assert bench.alu_peak_tflops(64, 152, 2070.0) == pytest.approx(1.2586, rel=1e-4)


def test_fp64_operator_entry_by_hand():
    peaks = {"bf16_tflops": 1982.0, "hbm_gbs": 6700.8}
    e = bench.roofline_entry("fp64_operator", 64, 7, 0.34733, CELLS, DOFS, 152, 2070.0, 1.056, peaks,
                             "not-the-sources", 4)
    flops = 12768 * CELLS
    ach = flops / 0.34733e-3 / 1e12
    assert e["flops_per_launch"] == flops
    assert e["achieved"] == pytest.approx(ach, abs=1e-4)
    assert e["peak"] == pytest.approx(1.2586, abs=1e-4)
    assert e["frac"] == pytest.approx(ach / 1.25856, abs=1e-4)
    assert e["frac_of_measured_fma"] == pytest.approx(ach / 1.056, abs=1e-4)
    # FP64 peak scaled from the measured bf16 burst by the nominal FP64 : dense bf16 ratio
    assert e["peak_from_measured_bf16"] == pytest.approx(1982.0 * 1.25856 / 2250.0, abs=1e-4)
    # 17 B per DoF (x read, y written, FP64) against the measured copy bandwidth
    assert e["algorithmic_bytes_per_launch"] == pytest.approx(17.0 * DOFS)
    assert e["hbm_frac_algorithmic"] == pytest.approx(17.0 * DOFS / 0.34733e-3 / 1e9 / 6700.8, abs=1e-4)
    # counters taken on other kernel sources are not reported
    assert e["traffic"] is None and "traffic_over_algorithmic_bytes" not in e


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha()
    assert len(sha) == 64
    rec = bench.traffic_record("fp64_operator", sha)
    committed = bench.json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))["fp64_operator"]
    if committed["kernel_source_sha256"] == sha:
        assert rec == committed["dram_bytes_per_launch_full_size"]
    else:
        assert rec is None
    assert bench.traffic_record("fp64_operator", "0" * 64) is None


def test_roofline_object_leads_with_the_largest_share():
    rl = {"a": {"frac": 0.5, "launch_list_share": 0.1}, "b": {"frac": 0.9, "launch_list_share": 0.3},
          "c": {"launch_list_share": 0.6}}  # no frac: cannot lead
    out = bench.roofline_object(rl, {"hbm_gbs": 6700.8}, "measured")
    assert out["key"] == "b" and out["frac"] == 0.9
    assert list(out["others"]) == ["c", "a"]
    assert out["hbm_peak_gbs"] == 6700.8
