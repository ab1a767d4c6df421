"""Host-side rules of bench.py: which clock records disqualify a timed region."""
import bench


def test_clock_rules():
    ok = {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]}
    assert bench.clock_problem(ok) is None
    assert bench.clock_problem({"sm_mhz": 1500.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]}) is None
    assert bench.clock_problem({"sm_mhz": 2000.0, "sm_max_mhz": 2070.0,
                                "reasons": ["hw_slowdown", "sw_power_cap"]}) == "hw_slowdown"
    assert bench.clock_problem({"sm_mhz": 2000.0, "sm_max_mhz": 2070.0,
                                "reasons": ["sw_thermal_slowdown"]}) == "sw_thermal_slowdown"
    # a clock held far below its maximum with no reason: a leftover lock
    assert "no reason" in bench.clock_problem({"sm_mhz": 1200.0, "sm_max_mhz": 2070.0, "reasons": []})
    assert bench.clock_problem({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}) is None


def test_traffic_figures_apply_only_to_the_captured_case():
    case = bench.GEMM_TRAFFIC_CASE
    got = bench.gemm_traffic("cgemm_expand", case["nr"], case["tile"], case["ranks"], case["precision"])
    # the committed sources either hash to the capture (a figure) or not (null)
    assert got is None or got == bench.GEMM_TRAFFIC_BYTES["cgemm_expand"]
    assert bench.gemm_traffic("cgemm_expand", case["nr"], case["tile"], case["ranks"][:-1],
                              case["precision"]) is None
    assert bench.gemm_traffic("cgemm_expand", case["nr"], 256, case["ranks"], case["precision"]) is None
    assert bench.gemm_traffic("cgemm_expand", case["nr"], case["tile"], case["ranks"], "fp32") is None


def test_rank_schedule_and_step_batches():
    wl = bench.PRECISION_FORM
    ranks = wl.ranks(wl.nfreq)
    assert ranks[0] == wl.rank_lo and ranks[-1] == wl.rank_hi and len(ranks) == 128
    assert all(b >= a for a, b in zip(ranks, ranks[1:]))
    from paper_2412_14973_gb300 import sharding
    steps = sharding.batches(sharding.frequency_plan(wl.nfreq, 0, 1), wl.batch)
    assert len(steps) == 16 and sorted(f for s in steps for f in s) == list(range(128))
    # every step spans the rank range (the captured traffic case is the first step)
    assert [ranks[f] for f in steps[0]] == bench.GEMM_TRAFFIC_CASE["ranks"]


def test_reference_arm_prints_one_contract_line():
    # the oracle as the reference arm: one bounded sample step, on the host
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--oracle-cols", "64"], capture_output=True, text=True, timeout=600,
                       cwd=root)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "freq-solves/s" and d["unit"] == "freq-solves/s"
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
