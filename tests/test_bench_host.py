"""Host logic of bench.py on CPU: the roofline rows computed from the
library's profiling counters, the clock record's parsing, and the reference
arm's JSON line (the FP64 oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2105_06975_gb300.wc4d import Stats  # noqa: E402


def _stats(**kw):
    st = Stats()
    for k, v in kw.items():
        setattr(st, k, v)
    return st


def test_kernel_rows_fractions_and_shares():
    hbm = 6795.8
    st = _stats(gemm_ms=700.0, gemm_flops=0.8e12, gemm_launches=2000,
                orth_ms=400.0, orth_bytes=1.6e12, orth_launches=1400)
    rows = bench.kernel_rows(st, step_ms=1000.0, hbm=hbm)
    g, o = rows["gemm_fp64"], rows["orth"]
    assert g["bound"] == "alu" and g["unit"] == "TFLOP/s"
    assert g["achieved"] == pytest.approx(0.8e12 / 0.7 / 1e12)
    assert g["frac"] == pytest.approx(g["achieved"] / bench.FP64_PEAK_TFLOPS)
    assert g["share_of_step"] == pytest.approx(0.7)
    assert g["flops_per_launch"] == pytest.approx(0.8e12 / 2000)
    assert o["bound"] == "hbm" and o["unit"] == "GB/s"
    assert o["achieved"] == pytest.approx(1.6e12 / 0.4 / 1e9)
    assert o["frac"] == pytest.approx(4000.0 / hbm)
    assert o["bytes_per_launch"] == pytest.approx(1.6e12 / 1400)
    assert "gemm_tc" not in rows and "gemm_df32" not in rows and "gemm_fp32" not in rows
    # no measured HBM peak: the fraction is left open rather than guessed
    assert bench.kernel_rows(st, 1000.0, hbm=None)["orth"]["frac"] is None


def test_orth_row_with_the_six_byte_basis():
    """orth_bytes count 8 B per basis entry (the FP64-equivalent floor the
    fraction uses); with the 6-byte basis the row adds what the passes move,
    and the roofline traffic is scaled from the 6-byte capture."""
    hbm = 6794.5
    st = _stats(orth_ms=100.0, orth_bytes=4e11, orth_moved_bytes=3e11, orth_launches=1000)
    o = bench.kernel_rows(st, step_ms=400.0, hbm=hbm, dcgs=True)["orth"]
    assert o["frac"] == pytest.approx(4000.0 / hbm)
    assert o["moved"]["achieved_gbs"] == pytest.approx(3000.0)
    assert o["moved"]["frac"] == pytest.approx(3000.0 / hbm)
    assert o["moved"]["bytes_per_launch"] == pytest.approx(3e8)
    assert "orth_b6" in bench.TRAFFIC_RATIO and 0.9 < bench.TRAFFIC_RATIO["orth_b6"][0] < 1.1
    # the 8-byte basis: no moved block (both counts agree)
    st8 = _stats(orth_ms=100.0, orth_bytes=4e11, orth_moved_bytes=4e11, orth_launches=1000)
    assert "moved" not in bench.kernel_rows(st8, 400.0, hbm=hbm, dcgs=True)["orth"]


def test_tensor_core_row_takes_the_tighter_roof(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"bf16_tflops": 1918.0})
    hbm = 6795.8
    # bytes-heavy launch: 3 TB/s of FP64-operator bytes (5.25 TB/s in the digit form) against 400 TF of
    # 1918 -> HBM is the tighter roof, measured on the FP64-operator floor
    st = _stats(gemmtc_ms=100.0, gemmtc_flops=1e9, gemmtc_bytes=5.25e11, gemmtc_alg_bytes=3e11,
                gemmtc_mma_flops=4e13, gemmtc_launches=10)
    r = bench.kernel_rows(st, 1000.0, hbm=hbm)["gemm_tc"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(3000.0 / hbm)
    assert r["bytes_per_launch"] == pytest.approx(3e10)
    assert r["digit_form"]["frac"] == pytest.approx(5250.0 / hbm)
    assert r["digit_form"]["bytes_per_launch"] == pytest.approx(5.25e10)
    assert r["tensor"]["frac"] == pytest.approx(400.0 / 1918.0)
    assert r["mma_flops_per_launch"] == pytest.approx(4e12)
    # flop-heavy launch: 1500 TF -> the tensor roof is the tighter one
    st.gemmtc_mma_flops = 1.5e14
    r = bench.kernel_rows(st, 1000.0, hbm=hbm)["gemm_tc"]
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1500.0) and r["peak"] == 1918.0


def test_clock_record_parsing():
    cs = bench.ClockSampler(0)
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.proc = Done()
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = cs.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    cs.lines.append("0, 1200, 2070, 700.0, 0x8, Not Active, Active, Not Active, Not Active")
    assert cs.stop()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


@pytest.mark.slow
def test_reference_arm_reports_only_full_solves():
    """The reference arm: every timed step is a full FP64 oracle solve of the
    scale window (s=2048, N=64, p=1024) on the host cores (about 30 s here);
    with the time budget spent after the first, it stops and reports one step
    (no modelled or extrapolated steps), its timed wall time covering it."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--ref-budget-s", "1"], capture_output=True, text=True,
                         timeout=900, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["steps_requested"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["ms_per_step"] == pytest.approx(1e3 / d["value"])
    # the claimed step time fits inside the measured wall time of the timed region
    assert d["steps"] * d["ms_per_step"] / 1e3 <= d["timed_wall_s"] * 1.0001
    assert d["config"]["s"] == 2048 and d["config"]["N"] == 64 and d["config"]["p"] == 1024
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    # the oracle meets the stopping rule the GPU solve uses
    assert cb["converged"] and cb["relres_true"] <= 1e-6 and 1 <= cb["iterations"] <= 1000
    assert "1 timed steps, each one full oracle solve" in cb["sample"] and "stopped after 1 of 2" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
