"""Host-side logic of bench.py, without a GPU: the roofline arithmetic of
the JSON line, the per-kind table of trapezoidal updates, the clock-sample
parsing that decides whether a run is kept, and the workload name."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _stats(total, kind_flops):
    return {"flops": [0.0, 0.0, 0.0, 0.0, total], "tpmqrt_kind_flops": kind_flops,
            "tpmqrt_kind_seconds": [1.0] * 8, "tpmqrt_kind": [1] * 8}


def test_roofline_fp64_is_the_alu_peak():
    peak = bench.FP64_PEAK_TFLOPS                # measured DFMA throughput
    assert 1.0 < peak < 1.3                      # GB300: 152 SMs x 2 DFMA/clk x 2 flop x <= 2.07 GHz
    r = bench.roofline(_stats(0.5 * peak * 1e12 * 10.0, [0.0] * 8), 10.0, True)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(peak) and r["achieved"] == pytest.approx(0.5 * peak)
    assert r["frac"] == pytest.approx(0.5)


def test_roofline_mixed_sums_tensor_and_simt_bound_times(monkeypatch):
    monkeypatch.setattr(bench, "TF32_PEAK_TFLOPS", 1100.0)
    monkeypatch.setattr(bench, "FP32_PEAK_TFLOPS", 80.0)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", "/nonexistent")
    p_tc = 1100.0 / 3.0                         # 3xTF32: three MMAs per algorithmic product
    p_simt = 80.0
    kinds = [1e12, 2e12, 30e12, 4e12, 5e12, 6e12, 7e12, 80e12]   # index = 4 Ydense + 2 Rdense + Adense
    total = sum(kinds) + 3e12                   # 3 TFLOP outside the updates (panels, T, ...)
    f_tc = kinds[2] + kinds[3] + kinds[5] + kinds[6] + kinds[7]
    t_bound = f_tc / (p_tc * 1e12) + (total - f_tc) / (p_simt * 1e12)
    r = bench.roofline(_stats(total, kinds), 2.0, False)
    assert r["bound"] == "tensor"
    assert r["frac"] == pytest.approx(t_bound / 2.0)
    assert r["peak"] == pytest.approx(total / t_bound / 1e12)
    assert r["achieved"] == pytest.approx(total / 2.0 / 1e12)
    assert r["tensor_part"]["tflop"] == pytest.approx(f_tc / 1e12)
    assert r["traffic"] is None
    # the kinds that stay on SIMT (Y low-rank with R low-rank, and Y dense
    # with both R and A low-rank) are not at the tensor rate
    assert f_tc == pytest.approx(127e12)


def test_tpmqrt_kind_names():
    st = {"tpmqrt_kind": [0, 0, 3, 0, 0, 0, 0, 5], "tpmqrt_kind_seconds": [0, 0, 1.5, 0, 0, 0, 0, 2.25],
          "tpmqrt_kind_flops": [0, 0, 2e9, 0, 0, 0, 0, 9e9]}
    out = bench.tpmqrt_kinds(st)
    assert set(out) == {"YL RD AL", "YD RD AD"}
    d = out["YD RD AD"]
    assert (d["n"], d["cta_s"], d["gflop"], d["pipe"]) == (5, 2.25, 9.0, "3xtf32")
    assert d["gflops_per_sm"] == pytest.approx(4.0)
    assert d["frac_of_sm_peak"] == pytest.approx(4.0 / (bench.TF32_PEAK_TFLOPS / 3 * 1e3 / 152), rel=1e-3)
    assert bench.tpmqrt_kinds(st, True)["YD RD AD"]["pipe"] == "fp64"


def test_traffic_only_for_the_captured_kernel(tmp_path, monkeypatch):
    f = tmp_path / "cap.md"
    f.write_text("# capture\n- csrc_sha16: " + bench.csrc_digest() + "\n- workload: small\n"
                 "- dram_bytes_per_counted_flop: 0.01\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    t, note = bench.dram_traffic(2e12)
    assert t == pytest.approx(2e10) and "small" in note
    f.write_text("- csrc_sha16: 0000000000000000\n- dram_bytes_per_counted_flop: 0.01\n")
    assert bench.dram_traffic(2e12)[0] is None


def test_extrapolation_uses_task_counts():
    sample = {"mean_task_s": {"geqrt": 1.0, "larfb": 2.0, "tsqrt": 3.0, "tpmqrt": 4.0}}
    p, q = 5, 3
    want = 3 * 1.0 + 3 * 2.0 + (4 + 3 + 2) * 3.0 + (4 * 2 + 3 * 1 + 0) * 4.0
    assert bench.extrapolate(sample, p, q) == pytest.approx(want)


def _sampler_with(lines):
    s = bench.ClockSampler(0)
    s.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0, kill=lambda: None)
    s.lines = lines
    return s


def test_clock_samples_median_and_reasons():
    ok = "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1900, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1200.0, 0x20, Not Active, Active, Not Active, Not Active"
    c = _sampler_with([ok, ok, capped]).stop()
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070 and c["reasons"] == ["sw_power_cap"]
    assert c["samples"] == 3
    c = _sampler_with([ok, hot, "garbage", ""]).stop()
    assert c["reasons"] == ["hw_thermal_slowdown"] and c["samples"] == 2
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_workload_name_names_sizes_and_variant():
    args = types.SimpleNamespace(size="full", tol=1e-5, ill_conditioned=False)
    name = bench.workload_name(args)
    assert "65536x32768" in name and "b=512" in name and "tol=1e-05" in name
    args.ill_conditioned = True
    assert bench.workload_name(args).endswith("columns scaled 1..1e-10")


def test_dense_equivalent_rate():
    m, n = 65536, 32768
    d = bench.dense_equivalent(m, n, 3.5)
    assert d["flop"] == pytest.approx(2 * m * n * n - 2 * n ** 3 / 3)
    assert d["tflops"] == pytest.approx(d["flop"] / 3.5 / 1e12)
    assert d["note"].startswith("context only")
    # square case: 4/3 n^3
    assert bench.dense_equivalent(3, 3, 1.0)["flop"] == pytest.approx(4 / 3 * 27)
