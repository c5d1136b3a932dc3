#!/usr/bin/env python3
"""Benchmark: interior-point time-to-solution for dynamical optimal transport.

One step = one complete interior-point solve (mu from 1 down to the first
stage with duality gap mu K/(K+1) <= 1e-6, Newton steps with FGMRES + BB) on
the workload of 64 x 64 squares (8192 coarse / 32768 fine triangles), K = 32,
rho_in / rho_f = seeded 3-Gaussian mixtures (seeds 2 / 3, floor 1e-4, unit
mass), inputs resident on the GPU.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Multi-GPU (torchrun, one rank per GPU): every rank solves its own replica of
the workload (the problem does not shard; replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "mix64"
WORKLOAD_DESC = ("64x64 squares -> 8192 coarse / 32768 fine triangles, K=32, 3-Gaussian mixtures "
                 "(centres U[0.15,0.85]^2, sigma U[0.05,0.15], weights U[0.5,1.5], seeds 2/3), floor 1e-4, "
                 "unit mass, mu0=1, mu <- mu/5, stop at duality gap 1e-6")
SAMPLE_N, SAMPLE_K = 12, 6   # bounded sample of the same density recipe for the CPU oracle
SAMPLE_EVERY = 16            # time one launch in 16 of the roofline kernel inside the timed region
METRIC = "IPM time-to-solution at duality gap 1e-6"
WORKLOAD_N, WORKLOAD_K = 64, 32


def workload_config(args, world: int) -> dict:
    """The config object both arms print (the reference arm times a bounded sample of this
    workload and names the sample in its cpu_baseline)."""
    n, K = WORKLOAD_N, WORKLOAD_K
    return {"workload": WORKLOAD_DESC, "precision": args.precision, "n": n, "K": K,
            "parallelism": f"replicas x{world}", "l2": "flushed between steps (256 MB write)",
            "unknowns": (K + 1) * 8 * n * n + K * 2 * n * n}
# dram__bytes_read.sum + dram__bytes_write.sum per launch, by kernel group, from an ncu capture of the
# kernel as it is built now; a group without an entry reports traffic None.  schur_line_smooth has none:
# its capture (profiles/k_line_pcr_tile_mix64.md, 1.372 MB per launch) predates the move of
# k_line_pcr_tile_kernel's body into inlined stage functions.
NCU_TRAFFIC: dict = {}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solves")
    p.add_argument("--no-batched", action="store_true", help="skip the 64-problem batched solve")
    p.add_argument("--batched-streams", type=int, default=16)
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return p.parse_args()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (every rank gets it); x itself at world size 1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n_items: int, rank: int, world: int) -> list:
    """Round-robin share of n_items independent problems for one rank (no exchange)."""
    return list(range(rank, n_items, world))


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ clocks
QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return summarise_clocks(lines)


def summarise_clocks(lines) -> dict | None:
    """Summary of nvidia-smi samples in the QUERY order (csv, no header, no units):
    median SM clock over the samples drawing at least half the peak power (the
    timed work), the maximum SM clock, and every throttle reason seen Active."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    pmax = max(r[2] for r in rows)
    load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[3][i].lower() == "active"})
    return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": reasons, "samples": len(rows), "power_w_max": pmax}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample_seconds() -> tuple[float, str]:
    """Time the oracle (single thread) on the bounded sample; runs in a child process."""
    code = ("import time,sys; sys.path.insert(0, %r)\n"
            "from oracle import ipm\nfrom ot_inputs import config_densities\n"
            "n,K,r0,r1 = config_densities('mixN', %d)\n"
            "d = ipm.discretise(n, %d)\nt = time.perf_counter()\nr = ipm.ipm_solve(d, r0, r1)\n"
            "print(time.perf_counter() - t, r.newton_steps)\n") % (ROOT, SAMPLE_N, SAMPLE_K)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    sec, steps = out.stdout.split()[-2:]
    desc = (f"oracle IPM (scipy SuperLU Newton solves, 1 thread) on the same density recipe at "
            f"{SAMPLE_N}x{SAMPLE_N} squares, K={SAMPLE_K} ({steps} Newton steps), one full solve; not extrapolated")
    return float(sec), desc


def run_reference(args, world, rank):
    if rank != 0:
        return
    times = []
    desc = ""
    for i in range(args.warmup + args.steps):
        t, desc = oracle_sample_seconds()
        if i >= args.warmup:
            times.append(t)
    v = sum(times) / len(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, world),
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our path
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from ot_inputs import config_densities
    from paper_2209_00315_gb300 import capi

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n, K, r0, r1 = config_densities(WORKLOAD)
    assert (n, K) == (WORKLOAD_N, WORKLOAD_K)
    mesh = capi.Mesh(n)
    r0d = torch.from_numpy(r0).to(dev)
    r1d = torch.from_numpy(r1).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed_solves(precision, steps, warmup, groups=None):
        opt = capi.default_options(precision=precision)
        for _ in range(warmup):
            capi.ot_ipm_solve(mesh, r0d, r1d, K, options=opt)
        barrier()
        if groups is not None:
            capi.ot_kernel_timing_enable(groups, sample_every=SAMPLE_EVERY)
        launches0 = capi.ot_kernel_launches()
        ms, res = [], None
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = capi.ot_ipm_solve(mesh, r0d, r1d, K, options=opt)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        barrier()
        launches = capi.ot_kernel_launches() - launches0
        timing = capi.ot_kernel_timing_read() if groups is not None else None
        if groups is not None:
            capi.ot_kernel_timing_enable(False)
        return ms, res, launches, timing

    # 1. which kernel group dominates (one untimed profiled solve, all groups on; per-launch
    #    events need the launches issued one by one, so this solve runs without graphs)
    eager = capi.default_options(precision=args.precision, graphs=0)
    capi.ot_ipm_solve(mesh, r0d, r1d, K, options=eager)
    capi.ot_kernel_timing_enable(True)
    capi.ot_ipm_solve(mesh, r0d, r1d, K, options=eager)
    torch.cuda.synchronize()
    prof_all = capi.ot_kernel_timing_read()
    capi.ot_kernel_timing_enable(False)
    dominant = max(prof_all, key=lambda k: prof_all[k][0])

    # 2. the timed region: only the dominant group carries events
    clocks = ClockSampler(local)
    ms, res, launches, timing = timed_solves(args.precision, args.steps, args.warmup, groups=[dominant])
    clk = clocks.stop()
    total = sum(ms)
    total = max_over_ranks(total, world, dev)
    sec = total / 1e3 / args.steps

    # 3. end to end through the public API with host buffers (copies inside the timed region)
    r0h = torch.from_numpy(r0).pin_memory()
    r1h = torch.from_numpy(r1).pin_memory()
    opt = capi.default_options(precision=args.precision)
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = capi.ot_ipm_solve(mesh, r0h, r1h, K, options=opt)
        t1 = time.perf_counter()
        e2e.append(t1 - t0)
    Np, Nr = (K + 1) * mesh.n_fine, K * mesh.n_coarse
    e2e_obj = {"value": sum(e2e) / len(e2e), "unit": "s", "h2d_bytes_per_step": 2 * mesh.n_coarse * 8,
               "d2h_bytes_per_step": (Np + 2 * Nr) * 8 + 8}

    # 4. FP64 GPU path for the mixed-vs-FP64 comparison of the metric
    fp64 = None
    if not args.no_fp64 and args.precision == "mixed":
        ms64, res64, _, _ = timed_solves("fp64", max(1, args.steps // 2 + 1), 1)
        fp64 = {"value": sum(ms64) / len(ms64) / 1e3, "unit": "s", "steps": len(ms64),
                "cost": res64["cost"], "newton_steps": res64["stats"]["newton_steps"],
                "fgmres_iters": res64["stats"]["fgmres_iters"]}

    # roofline of the dominant group, from the events of the timed region
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    t_ms, t_n, t_b = timing[dominant]
    achieved = (t_b / 1e9) / (t_ms / 1e3) if t_ms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(dominant),
                "launches": t_n, "avg_launch_us": 1e3 * t_ms / max(t_n, 1),
                "algorithmic_bytes_per_launch": t_b / max(t_n, 1),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"}

    # 5. the batched workload: 64 independent problems of uneven size on concurrent streams
    batched = None
    if not args.no_batched:
        from ot_inputs import batched_problem_specs

        specs_all = batched_problem_specs(64)
        specs = [specs_all[i] for i in shard(len(specs_all), rank, world)]
        bmeshes, items = {}, []
        for n_, K_, a_, b_ in specs:
            if n_ not in bmeshes:
                bmeshes[n_] = capi.Mesh(n_)
            items.append((bmeshes[n_], torch.from_numpy(a_).to(dev), torch.from_numpy(b_).to(dev), K_))
        bopt = capi.default_options(precision=args.precision)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bout = capi.ot_ipm_solve_batched(items, options=bopt, n_streams=args.batched_streams, raise_on_error=False)
        torch.cuda.synchronize()
        tb = max_over_ranks(time.perf_counter() - t0, world, dev)
        failed = [i for i, o in enumerate(bout) if o["status"] != 0]
        batched = {"workload": "64 problems, side in {16,24,32,48,64}, K in {8,16,24,32}, 1-4 Gaussians, "
                               "floor 1e-4 (seeds 1000..1063)",
                   "precision": args.precision, "n_streams": args.batched_streams, "seconds": tb,
                   "problems_per_s": len(specs_all) / tb, "converged": len(items) - len(failed),
                   "problems_this_rank": len(items),
                   "failed": {i: capi.STATUS.get(bout[i]["status"], bout[i]["status"]) for i in failed},
                   "newton_steps": sum(o["stats"]["newton_steps"] for o in bout),
                   "unknowns": sum((K_ + 1) * 8 * n_ * n_ + K_ * 2 * n_ * n_ for n_, K_, _, _ in specs)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, desc = oracle_sample_seconds()
        cpu = {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": desc}

    if rank != 0:
        return
    st = res["stats"]
    line = {
        "metric": METRIC,
        "value": sec, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": workload_config(args, world),
        "solves_per_s": world * args.steps / (total / 1e3),
        "newton_solves_per_s": world * st["newton_steps"] / sec,
        "result": {"cost": res["cost"], "newton_steps": st["newton_steps"], "fgmres_iters": st["fgmres_iters"],
                   "inner_iters": st["inner_iters"], "final_residual": st["final_residual"], "gap": st["gap"]},
        "fp64": fp64,
        "batched": batched,
        "speedup_mixed_vs_fp64": (fp64["value"] / sec) if fp64 else None,
        "e2e": e2e_obj,
        "gpu_launches": launches,
        "roofline": roofline,
        "kernel_share_ms_per_solve": {k: v[0] for k, v in prof_all.items()},
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
