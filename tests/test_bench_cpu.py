"""Host-side checks of bench.py: the reference arm's JSON line (it times the
FP64 oracle, no GPU involved), the roofline arithmetic and the traffic record
lookup."""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, HERE)

import bench  # noqa: E402


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(HERE, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=HERE)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["value"] == d["value"] and cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert isinstance(d["config"]["workload"], str)


@pytest.mark.parametrize("prec,n", [("bf16x2", 64), ("fp8", 64), ("bf16", 32)])
def test_roofline_hbm_forms(prec, n):
    """Tensor-core forms: 32 B per site-direction plus 16 B of coefficients
    per site, over the launch time, against the measured copy bandwidth."""
    sdu, t = 268435456, 1.6e-3
    r = bench._roofline(prec, n, sdu, t, {"hbm_gbs": 6500.0}, "measured")
    want = (32.0 + 16.0 / n) * sdu / t / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(want) and r["frac"] == pytest.approx(want / 6500.0)


def test_roofline_fp32_is_alu_bound():
    """The float32 CUDA-core form: 32 n flops per site-direction against the
    FP32 lanes x clock peak."""
    sdu, t, n = 268435456, 12.3e-3, 64
    r = bench._roofline("fp32", n, sdu, t, {"hbm_gbs": 6500.0, "sm_max_mhz": 2032.0}, "measured")
    peak = 148 * 128 * 2 * 2032e6 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(32.0 * n * sdu / t / 1e12)


def test_traffic_lookup():
    """An unrecorded kernel has no traffic; a recorded one scales its capture
    by sites when the sources still hash to the captured value (else None)."""
    assert bench._measured_traffic("no_such_kernel", 1000) is None
    with open(os.path.join(HERE, "profiles", "traffic.json")) as f:
        rec = json.load(f)["k_step_tc_pair"]
    got = bench._measured_traffic("k_step_tc_pair", 2 * rec["captured_sites"])
    if got is not None:
        assert got == pytest.approx(2 * (rec["dram_bytes_read"] + rec["dram_bytes_write"]))


def test_failing_leg_is_recorded_not_raised():
    def boom(x):
        raise RuntimeError(f"leg failed on {x}")
    assert bench._leg(lambda a, b: a + b, 2, 3) == 5
    assert bench._leg(boom, 7) == {"error": "RuntimeError: leg failed on 7"}
