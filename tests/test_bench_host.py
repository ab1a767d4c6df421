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
