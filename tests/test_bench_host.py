"""Host-side logic of bench.py on CPU: the clock record taken during the timed
region (median SM clock under load, the maximum, and every throttle reason
seen), and the throughput aggregation of one rank."""
import bench


def _write(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_clock_summary_takes_the_median_and_every_reason(tmp_path):
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    path = _write(tmp_path, [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "1, 500, 2070, 100.0, 0x8, Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line"])
    c = bench._clock_summary(path, 0)
    assert c["sm_mhz"] == 2070.0                # median of 2070, 1980, 2070
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]     # GPU 1's hw_slowdown is not ours
    assert c["samples"] == 3


def test_clock_summary_reports_a_throttled_run(tmp_path):
    path = _write(tmp_path, [
        "0, 1400, 2070, 1000.0, 0x40, Not Active, Active, Not Active, Not Active",
        "0, 1500, 2070, 1000.0, 0x20, Not Active, Not Active, Active, Not Active"])
    c = bench._clock_summary(path, 0)
    assert c["sm_mhz"] == 1450.0
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples(tmp_path):
    assert bench._clock_summary(str(tmp_path / "missing.csv"), 0)["reasons"] == ["unsampled"]
    assert bench._clock_summary(_write(tmp_path, ["1, 2070, 2070, 1, 0x0, a, b, c, d"]),
                                0)["reasons"] == ["unsampled"]


def test_kernel_source_hash_is_stable():
    assert bench._kernel_sources_sha() == bench._kernel_sources_sha()
    assert len(bench._kernel_sources_sha()) == 16
