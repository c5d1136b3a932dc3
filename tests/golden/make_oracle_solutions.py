#!/usr/bin/env python3
"""Write stored oracle solutions for the full-size parity tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``ot_inputs``): for each named workload it runs the interior-point method
with exact (sparse-LU) Newton directions, the paper's mu schedule
(mu <- mu/5 from 1, stop at the first stage with mu |Omega| K/(K+1) <= 1e-6,
Sec. 4.1) and the last stage solved to ||F|| <= 1e-11 max(1, ||F_0||), so
that the stored point is the unique barrier solution at the final mu to well
below the comparison tolerances (rho and s are unique for mu > 0, phi up to
one constant, Sec. 3.1, fixed here by zero M-weighted space-time mean).

  python tests/golden/make_oracle_solutions.py fd32        # 32x32 squares, K=16, seeds 6/7
  python tests/golden/make_oracle_solutions.py mixN:24     # 24x24 squares, K=12, seeds 2/3
  python tests/golden/make_oracle_solutions.py gauss_cube8 # 3D: 8^3 cubes, K=7 (test 4)

Output: tests/golden/<name>_oracle.npz with rho (K N'), phi ((K+1) N, gauged),
s (K N'), cost, dual, mu, newton_steps and the per-stage Newton counts.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import ipm  # noqa: E402
from ot_inputs import config_densities, cube_config_densities  # noqa: E402

FINAL_NEWTON_TOL = 1e-11


def write(name: str) -> str:
    """name: a workload of ot_inputs.config_densities, mixN:<n> (n x n squares, K = n/2), or
    a 3D workload of ot_inputs.cube_config_densities."""
    if name.startswith("mixN:"):
        n, K, r0, r1 = config_densities("mixN", int(name.split(":")[1]))
        name = f"mix{n}"
        d = ipm.discretise(n, K)
    elif name.startswith("gauss_cube"):
        n, K, r0, r1 = cube_config_densities(name)
        d = ipm.discretise_cube(n, K)
    else:
        n, K, r0, r1 = config_densities(name)
        d = ipm.discretise(n, K)
    t0 = time.perf_counter()
    res = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(final_newton_tol=FINAL_NEWTON_TOL))
    sec = time.perf_counter() - t0
    path = os.path.join(HERE, f"{name}_oracle.npz")
    np.savez_compressed(
        path,
        n=n, K=K,
        rho=res.rho, phi=ipm.phi_gauge(d, res.phi), s=res.s,
        cost=res.cost, dual=res.dual, mu=res.mu, newton_steps=res.newton_steps,
        stage_newton=np.array([st[1] for st in res.stages]),
        stage_residual=np.array([st[2] for st in res.stages]),
        final_newton_tol=FINAL_NEWTON_TOL,
    )
    print(f"{name}: n={n} K={K} cost={res.cost:.15e} dual={res.dual:.15e} mu={res.mu:.3e} "
          f"newton={res.newton_steps} {sec:.0f}s -> {path}", flush=True)
    return path


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["fd32"]:
        write(nm)
