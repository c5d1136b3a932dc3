"""Host logic of bench.py that needs no GPU: the summary of the nvidia-smi
clock samples taken during the timed region."""
import bench


def _row(sm, power, hw="Not Active", cap="Not Active", idx=0, smax=2070):
    return f"{idx}, {sm}, {smax}, {power}, 0x0000000000000000, {hw}, Not Active, Not Active, {cap}\n"


def test_clock_summary_uses_loaded_samples_and_collects_reasons():
    lines = [_row(2070, 120.0)] * 3 + [_row(1980, 400.0), _row(2010, 390.0, cap="Active"), _row(1995, 410.0)]
    s = bench.summarise_clocks(lines)
    assert s["sm_mhz"] == 1995 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 6 and s["power_w_max"] == 410.0


def test_clock_summary_flags_hardware_slowdown_and_skips_bad_lines():
    lines = ["garbage\n", "0, [N/A], 2070, 300, 0x0, Not Active, Not Active, Not Active, Not Active\n",
             _row(2070, 300.0), _row(1500, 310.0, hw="Active")]
    s = bench.summarise_clocks(lines)
    assert s["samples"] == 2 and s["reasons"] == ["hw_slowdown"]
    assert bench.summarise_clocks([]) is None and bench.summarise_clocks(["x\n"]) is None
