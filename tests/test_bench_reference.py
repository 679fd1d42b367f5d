"""The reference arm of bench.py (the CPU oracle, timed as it stands) on the CPU: one
timed step prints one JSON line with the keys the benchmark contract needs."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "site-updates/s (batched multispin shaken dynamics)"
    assert d["unit"] == "updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_oracle_sample_covers_every_size_with_equal_work():
    sys.path.insert(0, ROOT)
    import bench
    Ls, _, _ = bench.workload(0)
    plan = bench.oracle_sample_plan(Ls, 3)
    sizes = sorted(set(int(x) for x in Ls))
    assert sorted(set(L for L, _, _ in plan)) == sizes
    for L in sizes:
        groups = [g for LL, g, _ in plan if LL == L]
        assert len(groups) == min(3, sum(1 for x in Ls if int(x) == L))
        assert all(int(Ls[g]) == L for g in groups) and len(set(groups)) == len(groups)
    work = [L * L * steps for L, _, steps in plan]
    assert max(work) == min(work) == max(sizes) ** 2


def test_reference_sample_is_bounded_for_long_runs():
    sys.path.insert(0, ROOT)
    import bench
    Ls, _, _ = bench.workload(0)
    assert bench.reference_max_L(25) is None
    for n, cap in ((100, 256), (205, 128)):
        assert bench.reference_max_L(n) == cap
        plan = bench.oracle_sample_plan(Ls, 1, cap)
        assert max(L for L, _, _ in plan) == cap
        assert sorted(set(L for L, _, _ in plan)) == [L for L in (32, 64, 128, 256) if L <= cap]
        assert len(set(L * L * st for L, _, st in plan)) == 1


def test_roofline_calls_plus_planes_arithmetic():
    """The multispin roofline's bound: calls at the measured Philox rate plus 16 logic
    operations per call at the measured LOP3 rate, one after the other; and at the
    unit rates (20 wide products per call at 32 lanes/clk/SM, 36 logic operations per
    call at 64 lanes/clk/SM)."""
    sys.path.insert(0, ROOT)
    import bench
    sms, mhz = 152, bench.sm_max_mhz()
    clk = sms * mhz * 1e6
    rates = {"philox_calls": 1.0e11, "lop3": 4.0e12}
    calls, launch_s = 1.0e7, 2.0e-4
    r = bench.calls_plus_planes(calls, launch_s, rates, sms)
    meas = calls / 1.0e11 + 16 * calls / 4.0e12
    assert abs(r["bound_ms_measured_rates"] - meas * 1e3) < 1e-12
    assert abs(r["frac_measured_rates"] - meas / launch_s) < 1e-12
    unit = calls * 20 / (32 * clk) + calls * 36 / (64 * clk)
    assert abs(r["bound_ms_unit_rates"] - unit * 1e3) < 1e-12
    # the line's peak in calls/s is the same bound expressed as a rate
    peak = 1.0 / (1.0 / rates["philox_calls"] + bench.PLANE_OPS_PER_CALL / rates["lop3"])
    assert abs(calls / peak - meas) < 1e-15
