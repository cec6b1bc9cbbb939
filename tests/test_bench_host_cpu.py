"""Host logic of bench.py on the CPU: peak selection, roofline arithmetic,
choice of the dominant kernel category, and the parsing of the nvidia-smi
clock samples (throttle reasons decide whether a run is rejected)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PK = {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1800.0, "sm_max_mhz": 2070.0}


def test_peaks_by_bound_and_precision():
    bf, _ = bench._peak("tensor", "bf16", PK, "measured")
    assert bf == 1800.0                                   # sustained figure for kernels inside a long step
    tf, src = bench._peak("tensor", "tf32x3", PK, "measured")
    assert abs(tf - 1800.0 * 1.1 / 2.25) < 1e-9 and "1.1/2.25" in src
    no_sustained = {k: v for k, v in PK.items() if k != "bf16_tflops_sustained"}
    assert bench._peak("tensor", "bf16", no_sustained, "measured")[0] == 2000.0
    alu, _ = bench._peak("alu", "fp32", PK, "measured")
    assert abs(alu - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9          # 80.5 TFLOP/s
    assert bench._peak("alu", "fp64", PK, "measured")[0] == 1.25


def test_fallback_peaks_when_the_measured_file_is_absent(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk, src = bench.peaks()
    assert src == "fallback" and pk["hbm_gbs"] == 6800.0 and pk["bf16_tflops"] == 1900.0


def test_roofline_entry_arithmetic():
    c = {"launches": 10, "ms": 1.0, "flops": 1e10}
    r = bench.roofline_entry("site_layer", c, "tensor", "tf32x3", PK, "measured")
    assert abs(r["achieved"] - 10.0) < 1e-12                 # 1e9 flop per 100 us launch = 10 TFLOP/s
    assert abs(r["frac"] - 10.0 / (1800.0 * 1.1 / 2.25)) < 1e-12
    assert abs(r["avg_launch_us"] - 100.0) < 1e-9 and r["flops_per_launch"] == 1e9
    assert r["mma_passes"] == 3 and r["unit"] == "TFLOP/s"
    assert r["traffic"] == bench.NCU_TRAFFIC[(bench.WORKLOAD, "tf32x3", "site_layer")]
    assert bench.roofline_entry("site_layer", c, "tensor", "tf32", PK, "measured")["traffic"] is None
    assert bench.roofline_entry("site_layer", {"launches": 0, "ms": 0.0, "flops": 0.0}, "tensor", "tf32x3",
                                PK, "measured") is None


def test_roofline_reports_the_longest_category_with_a_flop_model():
    prof = {"half_system_product": {"launches": 4, "ms": 2.0, "flops": 8e9},
            "site_layer": {"launches": 12, "ms": 3.0, "flops": 6e9},
            "subspace_gemm": {"launches": 8, "ms": 1.0, "flops": 1e9},
            "projector_svd": {"launches": 50, "ms": 9.0, "flops": 0.0}}      # no flop model: never chosen
    main, tc = bench.roofline_for("tf32x3", prof, PK, "measured")
    assert main["kernel"] == "site_layer" and main["bound"] == "tensor"
    assert tc["kernel"] == "site_layer"
    main32, tc32 = bench.roofline_for("fp32", prof, PK, "measured")
    assert main32["bound"] == "alu" and tc32 is None


def test_roofline_on_the_measured_bench_profile():
    """Category times of a default bench run on one GB300 (5 timed steps);
    flops of the CholQR2 category from its model 5 n k^2 + 2 n k + 2 k^3 / 3
    at n = 1024, k = 80 per call."""
    n, k, calls = 1024, 80, 1040
    prof = {"projector_svd": {"launches": 520, "ms": 275.996, "flops": 0.0},
            "cholqr_orth": {"launches": calls, "ms": 108.986,
                            "flops": calls * (5.0 * n * k * k + 2.0 * n * k + 2.0 * k ** 3 / 3.0)},
            "absorb": {"launches": 520, "ms": 51.933, "flops": 0.0},
            "corners": {"launches": 520, "ms": 45.647, "flops": 0.0},
            "als_gauge": {"launches": 25, "ms": 41.958, "flops": 0.0},
            "svd_jacobi": {"launches": 520, "ms": 41.714, "flops": 1029.0},
            "site_layer": {"launches": 1560, "ms": 31.019, "flops": 837518622720.0},
            "subspace_gemm": {"launches": 1040, "ms": 24.917, "flops": 174483046400.0},
            "half_system_product": {"launches": 520, "ms": 15.782, "flops": 1116691496960.0},
            "metric": {"launches": 40, "ms": 5.183, "flops": 0.0}}
    main, tc = bench.roofline_for("tf32x3", prof, PK, "measured")
    assert main["kernel"] == "cholqr_orth" and main["bound"] == "alu" and main["traffic"] is None
    assert 0.3 < main["achieved"] < 0.34 and main["frac"] < 0.005          # ~0.32 TFLOP/s: latency-bound
    assert tc["kernel"] == "site_layer" and abs(tc["achieved"] - 27.0) < 0.1


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.f = open(s.path, "w")
    s.f.write("\n".join(lines) + "\n")
    s.f.flush()
    s.proc = _Done()
    return s


def test_clock_samples_median_and_reasons(tmp_path):
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",   # unparsable: skipped
             "garbage"]
    r = _sampler_with(tmp_path, lines).stop()
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_samples_flag_thermal_slowdown(tmp_path):
    lines = ["0, 1500, 2070, 1200.0, 0x40, Not Active, Active, Not Active, Not Active",
             "0, 1400, 2070, 1200.0, 0x88, Active, Not Active, Active, Not Active"]
    r = _sampler_with(tmp_path, lines).stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1450.0


def test_no_samples_gives_no_clock_record(tmp_path):
    assert _sampler_with(tmp_path, ["garbage"]).stop() is None
    s = bench.ClockSampler(0)
    s.proc = None
    assert s.stop() is None


@pytest.mark.parametrize("ctm,obs,want", [(4, 2, 26), (1, 1, 8)])
def test_sweeps_per_step(ctm, obs, want):
    class A:
        ctm_sweeps, obs_sweeps = ctm, obs
    assert bench.sweeps_per_step(A) == want
