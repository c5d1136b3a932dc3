"""Captured (CUDA-graph) Krylov cycles against the same kernels launched one by one.

With ot_options.graphs = 1 every FGMRES cycle of a Newton step, the inner
Schur solves of its BB preconditioner applications included, runs as one CUDA
graph whose loops are conditional WHILE nodes; with graphs = 0 the same
kernels are launched one at a time and the host reads the convergence state
after every Krylov step.  Both orders of work are identical, so the results
must agree to FP64 rounding (1e-12 relative), with the same iteration counts
and the same number of kernel launches.
"""
import numpy as np
import pytest
import torch

from ot_inputs import config_densities

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = b.detach().cpu().numpy() if isinstance(b, torch.Tensor) else np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,precision", [(10, "mixed"), (16, "mixed"), (12, "fp64")])
def test_captured_solve_equals_uncaptured(gpu_lib, n, precision):
    from paper_2209_00315_gb300 import capi

    _, K, r0, r1 = config_densities("mixN", n)
    mesh = capi.Mesh(n)
    r0d, r1d = torch.from_numpy(r0).to(DEV), torch.from_numpy(r1).to(DEV)
    out = {}
    for g in (0, 1):
        opt = capi.default_options(precision=precision, graphs=g)
        capi.ot_ipm_solve(mesh, r0d, r1d, K, options=opt)  # workspace, graphs and shared memory set up
        torch.cuda.synchronize()
        l0 = capi.ot_kernel_launches()
        res = capi.ot_ipm_solve(mesh, r0d, r1d, K, options=opt)
        torch.cuda.synchronize()
        out[g] = (res, capi.ot_kernel_launches() - l0)
    (a, la), (b, lb) = out[0], out[1]
    assert a["stats"]["newton_steps"] == b["stats"]["newton_steps"]
    assert a["stats"]["fgmres_iters"] == b["stats"]["fgmres_iters"]
    assert a["stats"]["inner_iters"] == b["stats"]["inner_iters"]
    assert abs(a["cost"] - b["cost"]) <= 1e-12 * abs(a["cost"])
    for key in ("rho", "phi", "s"):
        assert rel(b[key], a[key]) < 1e-12, key
    # the graph's launch accounting (captured nodes times loop trips) counts the eager launches
    assert la == lb, (la, lb)


def test_captured_newton_direction_equals_uncaptured(gpu_lib):
    from paper_2209_00315_gb300 import capi

    n, K, r0, r1 = 8, 8, *config_densities("mixN", 8)[2:]
    mesh = capi.Mesh(n)
    r0d, r1d = torch.from_numpy(r0).to(DEV), torch.from_numpy(r1).to(DEV)
    # an interior state: the solution of the second barrier stage (mu = 0.2), then a step of the next
    res = capi.ot_ipm_solve(mesh, r0d, r1d, K, tol=0.5, options=capi.default_options(precision="mixed"))
    mu = 0.04
    dirs = {}
    for g in (0, 1):
        opt = capi.default_options(precision="mixed", graphs=g)
        dirs[g] = capi.ot_newton_solve(mesh, K, mu, res["phi"], res["rho"], res["s"], r0d, r1d, options=opt)
    for i in range(3):
        assert rel(dirs[1][i], dirs[0][i]) < 1e-12, i
    assert dirs[0][3]["fgmres_iters"] == dirs[1][3]["fgmres_iters"]


@pytest.mark.parametrize("graphs", [0, 1])
def test_programmatic_dependent_launch_changes_nothing(gpu_lib, graphs):
    """ot_options.pdl lets each kernel be scheduled while its predecessor's last
    blocks finish; every kernel first waits for its predecessor's results, so
    the iterates are bitwise those of plain stream order, captured or not."""
    from paper_2209_00315_gb300 import capi

    n = 16
    _, K, r0, r1 = config_densities("mixN", n)
    mesh = capi.Mesh(n)
    r0d, r1d = torch.from_numpy(r0).to(DEV), torch.from_numpy(r1).to(DEV)
    out = {}
    for pdl in (0, 1):
        opt = capi.default_options(precision="mixed", graphs=graphs, pdl=pdl)
        out[pdl] = capi.ot_ipm_solve(mesh, r0d, r1d, K, options=opt)
    a, b = out[0], out[1]
    assert a["stats"]["fgmres_iters"] == b["stats"]["fgmres_iters"]
    assert a["stats"]["inner_iters"] == b["stats"]["inner_iters"]
    assert a["cost"] == b["cost"]
    for key in ("rho", "phi", "s"):
        assert torch.equal(a[key], b[key]), key
