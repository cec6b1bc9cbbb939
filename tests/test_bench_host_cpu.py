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
    r = bench.roofline_entry("corners", c, "tensor", "tf32x3", PK, "measured")
    assert abs(r["achieved"] - 10.0) < 1e-12                 # 1e9 flop per 100 us launch = 10 TFLOP/s
    assert abs(r["frac"] - 10.0 / (1800.0 * 1.1 / 2.25)) < 1e-12
    assert abs(r["avg_launch_us"] - 100.0) < 1e-9 and r["flops_per_launch"] == 1e9
    assert r["mma_passes"] == 3 and r["unit"] == "TFLOP/s"
    assert r["traffic"] is None                                # no stored DRAM counters
    assert bench.roofline_entry("corners", {"launches": 0, "ms": 0.0, "flops": 0.0}, "tensor", "tf32x3",
                                PK, "measured") is None


def test_roofline_is_the_enlarged_corner_step():
    """The main entry is the two enlarged corners of a move, by their
    algorithmic (layered) flop count; categories without a flop model are
    never reported."""
    D, chi, p = 4, 64, 16
    per_move = 2 * (2 * chi ** 3 * D ** 2 + 2 * chi ** 3 * D ** 4 + 4 * p * chi ** 2 * D ** 6)
    prof = {"corners": {"launches": 520, "ms": 45.647, "flops": 520 * per_move},
            "half_system_product": {"launches": 520, "ms": 15.782, "flops": 1116691496960.0},
            "cholqr_orth": {"launches": 1040, "ms": 108.986, "flops": 1040 * 3.3273e7},
            "projector_svd": {"launches": 520, "ms": 275.996, "flops": 0.0}}
    r = bench.roofline_for("tf32x3", prof, PK, "measured")
    assert r["corners"]["bound"] == "tensor" and r["corners"]["kernel"] == "corners"
    assert abs(r["corners"]["flops_per_launch"] - per_move) < 1.0
    assert abs(r["corners"]["achieved"] - per_move / 87.78e-6 / 1e12) < 0.01
    assert r["cholqr_orth"]["bound"] == "alu" and "projector_svd" not in r
    r32 = bench.roofline_for("fp32", prof, PK, "measured")
    assert r32["corners"]["bound"] == "alu"


def test_step_flop_model():
    """F_move = 8 chi^3 D^4 + 12 p chi^2 D^6 + 2 chi^3 D^6, four moves a sweep:
    2.4e10 flops per sweep at (D, chi) = (4, 64) and 2.0e12 at (6, 144)."""
    assert abs(bench.step_flops(4, 64, 1) / 2.4e10 - 1.0) < 0.02
    assert abs(bench.step_flops(6, 144, 1) / 2.0e12 - 1.0) < 0.02
    assert bench.step_flops(4, 64, 26) == 26 * bench.step_flops(4, 64, 1)


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
