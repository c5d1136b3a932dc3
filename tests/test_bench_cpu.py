"""Host logic of bench.py that needs no GPU: the summary of the nvidia-smi
clock samples taken during the timed region, and the reference arm (the CPU
oracle on its bounded sample) and its JSON line."""
import numpy as np

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
    """The reference arm times the oracle's Newton steps on its bounded samples (warm-up
    runs discarded), extrapolates to the workload, prints one JSON line on rank 0 with
    the same metric, unit and config as the GPU arm, and nothing on other ranks."""
    import json

    # per-step times (n=16, n=24) of three runs: warm-up, then two timed steps, then the all-cores run
    runs = iter([[(16, 8, 9.0), (24, 12, 90.0)], [(16, 8, 1.0), (24, 12, 10.0)], [(16, 8, 1.0), (24, 12, 10.0)],
                 [(16, 8, 0.5), (24, 12, 5.0)]])
    monkeypatch.setattr(bench, "oracle_newton_seconds", lambda threads, samples=None: next(runs))
    bench.run_reference(_args(), 1, 0)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "s"
    assert line["higher_is_better"] is False
    assert line["config"] == bench.workload_config(_args(), 1)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["extrapolated"] is True and cb["cores"] == 1
    # per-step time 10 s at 24x24, K=12, growing as unknowns^p with 10x over the step from n=16
    u16, u24, uw = bench.unknowns(16, 8), bench.unknowns(24, 12), bench.unknowns(64, 32)
    p = np.log(10.0) / np.log(u24 / u16)
    expect = 10.0 * (uw / u24) ** p * bench.WORKLOAD_NEWTON_STEPS
    assert abs(line["value"] - expect) < 1e-9 * expect and abs(cb["value"] - expect) < 1e-9 * expect
    assert "64x64, K=32" in cb["sample"] and "extrapolated" in cb["sample"]
    assert line["cpu_baseline_all_cores"]["per_newton_step_s"] > 0
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    bench.run_reference(_args(), 2, 1)
    assert capsys.readouterr().out == ""


def test_baseline_fit_over_three_sizes(monkeypatch):
    """Three sample sizes on an exact power law t = a u^2 give p = 2 and the power law's value at
    the workload's unknown count."""
    u = bench.unknowns
    pts = [(n, n // 2, 1e-9 * u(n, n // 2) ** 2) for n in (12, 18, 24)]
    monkeypatch.setattr(bench, "oracle_newton_seconds", lambda threads, samples=None: pts)
    b = bench.oracle_baseline(1, newton_steps=10)
    assert abs(b["growth_exponent"] - 2.0) < 1e-9
    assert abs(b["per_newton_step_s"] - 1e-9 * u(64, 32) ** 2) < 1e-6 * b["per_newton_step_s"]
    assert abs(b["value"] - 10 * b["per_newton_step_s"]) < 1e-9 * b["value"]


def test_unknowns_of_the_newton_system():
    """(K+1) N + 2 K N' with N = 8 n^2, N' = 2 n^2: 1,605,632 for 64x64, K = 32 (phi, rho and s)."""
    assert bench.unknowns(64, 32) == 33 * 32768 + 2 * 32 * 8192 == 1605632


def test_oracle_sample_runs_in_a_child_process():
    """The child process that times the oracle's Newton steps finishes and reports each size."""
    pts = bench.oracle_newton_seconds(1, samples=[(4, 1), (6, 1)])
    assert [(n, K) for n, K, _ in pts] == [(4, 4), (6, 4)] and all(0 < t < 60 for _, _, t in pts)
