"""Command-line solve of one synthetic transport problem.

    python -m paper_2209_00315_gb300.solve --workload mix64 --precision mixed

runs the interior-point method (Sec. 3) on the GPU for a named seeded
workload of ``ot_inputs`` and prints one JSON line with the cost, the
iteration counts and the wall time of each solve.  Workloads: gauss8
(8x8, K=8), mix64 (64x64, K=32), mix128 (128x128, K=32), fd32 (32x32,
K=16), stress256 (256x256, K=64).
"""
import argparse
import json
import time

import torch

from . import capi


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--workload", default="mix64")
    p.add_argument("--n", type=int, default=None, help="squares per side for --workload mixN (K = n/2)")
    p.add_argument("--max-newton", type=int, default=None, help="Newton steps per barrier stage")
    p.add_argument("--allow-unconverged", action="store_true",
                   help="report a Newton or FGMRES cap as a result (exit 0), e.g. to profile a few capped steps")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--repeat", type=int, default=1)
    p.add_argument("--tol", type=float, default=1e-6, help="duality-gap target")
    p.add_argument("--verbose", action="store_true", help="print one line per barrier stage")
    p.add_argument("--restart", type=int, default=None, help="FGMRES restart length")
    p.add_argument("--max-iter", type=int, default=None, help="FGMRES iteration cap per Newton step")
    p.add_argument("--mu-factor", type=float, default=None, help="barrier reduction per stage (default 0.2)")
    p.add_argument("--graphs", type=int, choices=[0, 1], default=None,
                   help="1: FGMRES cycles as captured CUDA graphs (default); 0: launches one by one")
    p.add_argument("--gs-shadow", type=int, choices=[0, 1], default=None,
                   help="1: Gram-Schmidt dots from the FP32 basis copy (default); 0: all FP64")
    p.add_argument("--K", type=int, default=None, help="time steps, overriding the workload's K")
    p.add_argument("--precond", choices=["bb", "simple", "hybrid"], default=None,
                   help="outer preconditioner (default bb); hybrid: SIMPLE for mu < --simple-mu")
    p.add_argument("--simple-mu", type=float, default=None, help="hybrid switch (default 1e-5)")
    p.add_argument("--smooth-sweeps", type=int, default=None, help="multigrid pre/post sweeps per level")
    p.add_argument("--coarse-sweeps", type=int, default=None, help="multigrid sweeps on the coarsest level")
    p.add_argument("--lap-cycles", type=int, default=None, help="V-cycles per slice-Laplacian solve")
    p.add_argument("--pdl", type=int, choices=[0, 1], default=None,
                   help="1: programmatic dependent launch (default); 0: plain stream order")
    a = p.parse_args(argv)

    from ot_inputs import config_densities

    n, K, r0, r1 = config_densities(a.workload, a.n) if a.workload == "mixN" else config_densities(a.workload)
    if a.K is not None:
        K = a.K
    mesh = capi.Mesh(n)
    r0d = torch.from_numpy(r0).cuda()
    r1d = torch.from_numpy(r1).cuda()
    extra = {}
    if a.restart is not None:
        extra["fgmres_restart"] = a.restart
    if a.max_iter is not None:
        extra["fgmres_max_iter"] = a.max_iter
    if a.mu_factor is not None:
        extra["mu_factor"] = a.mu_factor
    if a.graphs is not None:
        extra["graphs"] = a.graphs
    if a.gs_shadow is not None:
        extra["gs_shadow"] = a.gs_shadow
    if a.max_newton is not None:
        extra["max_newton"] = a.max_newton
    if a.precond is not None:
        extra["precond"] = a.precond
    if a.simple_mu is not None:
        extra["simple_mu"] = a.simple_mu
    for f in ("smooth_sweeps", "coarse_sweeps", "lap_cycles", "pdl"):
        if getattr(a, f) is not None:
            extra[f] = getattr(a, f)
    opt = capi.default_options(precision=a.precision, verbose=int(a.verbose), **extra)
    walls, res = [], None
    for _ in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            res = capi.ot_ipm_solve(mesh, r0d, r1d, K, tol=a.tol, options=opt)
        except capi.OTError as e:
            if not (a.allow_unconverged and e.code == 4):
                raise
            torch.cuda.synchronize()
            print(json.dumps({"workload": a.workload, "n": n, "K": K, "stopped": str(e)}))
            return
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
    st = res["stats"]
    print(json.dumps({
        "workload": a.workload, "n": n, "K": K, "precision": a.precision, "cost": res["cost"],
        "newton_steps": st["newton_steps"], "fgmres_iters": st["fgmres_iters"], "inner_iters": st["inner_iters"],
        "gap": st["gap"], "wall_s": walls, "kernel_launches": capi.ot_kernel_launches(),
        "fgmres_restart": opt.fgmres_restart, "fgmres_max_iter": opt.fgmres_max_iter,
        "mu_factor": opt.mu_factor, "mu_final": st["mu"], "graphs": opt.graphs, "gs_shadow": opt.gs_shadow,
        "precond": ["bb", "simple", "hybrid"][opt.precond], "simple_mu": opt.simple_mu,
        "smooth_sweeps": opt.smooth_sweeps, "coarse_sweeps": opt.coarse_sweeps, "lap_cycles": opt.lap_cycles,
        "pdl": opt.pdl,
        "stage_newton": st["stage_newton"], "stage_outer": st["stage_outer"], "stage_inner": st["stage_inner"],
        "stage_seconds": st["stage_seconds"],
    }))


if __name__ == "__main__":
    main()
