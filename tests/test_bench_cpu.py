"""Host logic of bench.py that needs no GPU: the summary of the nvidia-smi
clock samples taken during the timed region, and the reference arm (the CPU
oracle on its bounded sample) and its JSON line."""
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


def _args(**kw):
    import argparse

    base = dict(gpus=1, steps=2, warmup=1, impl="reference", precision="mixed")
    base.update(kw)
    return argparse.Namespace(**base)


def test_reference_arm_prints_one_line_with_the_workload_config(monkeypatch, capsys):
    """The reference arm times the oracle on its bounded sample (warm-up runs
    discarded), prints one JSON line on rank 0 with the same metric, unit and config
    as the GPU arm, and nothing on other ranks."""
    import json

    times = iter([9.0, 2.0, 4.0])
    monkeypatch.setattr(bench, "oracle_sample_seconds", lambda: (next(times), "a bounded sample"))
    bench.run_reference(_args(), 1, 0)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "s"
    assert line["value"] == 3.0 and line["higher_is_better"] is False
    assert line["config"] == bench.workload_config(_args(), 1)
    assert line["cpu_baseline"] == {"value": 3.0, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": "a bounded sample"}
    assert line["e2e"] == {"value": 3.0, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    bench.run_reference(_args(), 2, 1)
    assert capsys.readouterr().out == ""


def test_oracle_sample_runs_in_a_child_process():
    """The child process that times the oracle sample finishes and reports its Newton steps."""
    sec, desc = bench.oracle_sample_seconds()
    assert 0 < sec < 600 and "Newton steps" in desc and f"{bench.SAMPLE_N}x{bench.SAMPLE_N}" in desc
