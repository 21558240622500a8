"""Host-side pieces of the benchmark line: the clock record, from
nvidia-smi rows sampled during the timed region (median SM clock, maximum
clock, and every throttle reason seen active; a run with a hardware or
thermal slowdown is not a valid measurement, sw_power_cap is kept and
noted), and the roofline's DRAM traffic read from the committed ncu
summary."""

from bench import ClockSampler


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", sm, mx, "900.0", "0x0", hw, hwt, swt, cap]


def test_summary_median_max_and_reasons():
    c = ClockSampler(0)
    c.rows = [_row("2070", "2070"), _row("1980", "2070", cap="Active"), _row("2055", "2070"),
              _row("[N/A]", "[N/A]"), _row("2070", "2070", hwt="active")]
    s = c.summary()
    assert s["sm_mhz"] == 2062.5            # median of the four readable samples
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["samples"] == 5


def test_summary_without_samples():
    s = ClockSampler(0).summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["no samples"]


def test_traffic_comes_from_the_committed_profile():
    """roofline.traffic is the trailing kernel's ncu DRAM bytes per tile
    (profiles/slice_gemm_trail_C1_B8.md) times the tiles of a launch."""
    from bench import _traffic_per_launch
    per_tile = _traffic_per_launch(1.0)
    assert per_tile is not None
    # the working matrix's read and write: 128 x 64 complex double-float = 262 KB
    assert 262_144 <= per_tile <= 1.05 * 262_144
