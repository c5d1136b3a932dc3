"""The stored oracle solutions of the full-size GPU parity tests, checked on the CPU.

tests/golden/<name>_oracle.npz is written by tests/golden/make_oracle_solutions.py
(the oracle's interior-point method with exact Newton steps, the last stage to
||F|| <= 1e-11).  These checks use the oracle's residual, cost and dual value
at the stored point, so a stale or truncated file fails here, on the CPU.
"""
import os

import numpy as np
import pytest

from oracle import ipm
from ot_inputs import config_densities, cube_config_densities

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# stored file -> the workload it was solved on (ot_inputs.config_densities arguments; the 3D
# workload of the paper's test 4 through cube_config_densities)
STORED = {"fd32": ("fd32",), "mix24": ("mixN", 24), "gauss_cube8": ("gauss_cube8",)}


def _workload(name):
    if name.startswith("gauss_cube"):
        n, K, r0, r1 = cube_config_densities(*STORED[name])
        return n, K, r0, r1, ipm.discretise_cube(n, K)
    n, K, r0, r1 = config_densities(*STORED[name])
    return n, K, r0, r1, ipm.discretise(n, K)


@pytest.mark.parametrize("name", sorted(STORED))
def test_stored_solution_is_a_converged_oracle_point(name):
    """At the stored point the oracle's residual meets the final tolerance,
    masses match rho_in slice by slice, rho and s are positive, the cost
    recomputes, the duality gap is the barrier's mu |Omega| K/(K+1) (Eq. 3.9 at
    a solution of the barrier problem) and phi carries the zero-mean gauge."""
    g = np.load(os.path.join(GOLDEN, f"{name}_oracle.npz"))
    n, K, r0, r1, d = _workload(name)
    assert (n, K) == (int(g["n"]), int(g["K"]))
    phi, rho, s, mu = g["phi"], g["rho"], g["s"], float(g["mu"])
    F = ipm.residual(d, phi, rho, s, r0, r1, mu)
    assert ipm.residual_norm(F) < 1e-10
    area = d.t.coarse.area
    assert np.abs(d.rho_slices(rho) @ area - area @ r0).max() < 1e-12
    assert rho.min() > 0 and s.min() > 0
    c = ipm.cost(d, phi, rho, r0, r1)
    assert abs(c - float(g["cost"])) < 1e-13 * c
    gap = mu * area.sum() * K / (K + 1)
    assert abs((c - ipm.dual_value(d, phi, r0, r1)) - gap) < 1e-6 * gap
    assert abs(np.tile(d.t.fine.area, K + 1) @ phi) < 1e-12
    # the stages follow the paper's schedule mu <- mu / 5 from 1 (Sec. 4.1)
    assert abs(mu - 0.2 ** (len(g["stage_newton"]) - 1)) < 1e-15
