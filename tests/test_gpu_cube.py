"""The 3D Cartesian variant's operators on the GPU against the oracle (needs a GPU).

Test 4 of Sec. 4.1 on n^3 cubes with J = I: the residual F (Eq. conservation,
hj and ortho discrete), the projected KKT operator [A, B^T P^T; P B, -P C P^T]
and the cost and dual value (reading R15), computed by the library's cube
kernels through the C ABI, against the oracle's sparse operators on the same
cube grid (`ipm.discretise_cube`) at seeded random states.  Both sides are
FP64 evaluations of the same sums in another order: 1e-13 relative.  Sizes
from one cube to 9^3 (729 cells, several thread blocks with a ragged tail).
"""
import numpy as np
import pytest
import torch

from oracle import ipm

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
# the oracle's projection P is assembled as a dense block per slice, so its KKT operator grows
# as N'^2: 9^3 keeps it to seconds (17^3, run once on the GB300, took the oracle minutes)
SIZES = [(1, 1), (2, 3), (3, 2), (5, 4), (8, 3), (9, 3)]


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def state(d, seed):
    rng = np.random.default_rng(seed)
    phi = 0.3 * rng.standard_normal((d.K + 1) * d.N)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    rho = ipm.renormalise(d, rng.uniform(0.5, 2, d.K * d.Nc), r0)
    s = rng.uniform(0.5, 2, d.K * d.Nc)
    return phi, rho, s, r0, r1


@pytest.fixture(scope="module", params=SIZES, ids=[f"{n}^3-K{K}" for n, K in SIZES])
def case(request, gpu_lib):
    from paper_2209_00315_gb300 import capi

    n, K = request.param
    d = ipm.discretise_cube(n, K)
    return n, K, d, capi.Mesh(n, kind="cube"), state(d, 13 * n + K)


def test_cube_residual_matches_oracle(case):
    from paper_2209_00315_gb300 import capi

    n, K, d, mesh, (phi, rho, s, r0, r1) = case
    mu = 0.23
    Fphi, Frho, Fs, norms = capi.ot_residual(mesh, K, mu, T(phi), T(rho), T(s), T(r0), T(r1))
    ref = ipm.residual(d, phi, rho, s, r0, r1, mu)
    assert rel(Fphi, ref[0]) < 1e-13 and rel(Frho, ref[1]) < 1e-13 and rel(Fs, ref[2]) < 1e-13
    assert abs(norms[3] - ipm.residual_norm(ref)) < 1e-12 * ipm.residual_norm(ref)


def test_cube_projected_kkt_operator_matches_oracle(case):
    from paper_2209_00315_gb300 import capi

    n, K, d, mesh, (phi, rho, s, r0, r1) = case
    x = np.random.default_rng(5 + n).standard_normal((K + 1) * d.N + K * d.Nc)
    y = capi.ot_kkt_apply(mesh, K, T(phi), T(rho), T(s), T(r0), T(r1), T(x))
    ref = d.projected_kkt(phi, rho, s, r0, r1) @ x
    assert rel(y, ref) < 1e-13


def test_cube_cost_and_dual_match_oracle(case):
    from paper_2209_00315_gb300 import capi

    n, K, d, mesh, (phi, rho, s, r0, r1) = case
    c, dv = capi.ot_cost_dual(mesh, K, T(phi), T(rho), T(r0), T(r1))
    ref_c = ipm.cost(d, phi, rho, r0, r1)   # 0 on a single cube: no interior face
    assert abs(c - ref_c) <= 1e-13 * abs(ref_c)
    ref = ipm.dual_value(d, phi, r0, r1)
    assert abs(dv - ref) <= 1e-13 * max(abs(ref), 1.0)


def test_cube_operators_at_the_oracle_solution_of_the_3d_gaussians(gpu_lib):
    """At the stored oracle solution of the 3D Gaussian test (8^3 cubes, K = 7, last
    stage to 1e-11) the GPU residual is at the oracle's level and the GPU cost
    and dual value give the barrier gap mu |Omega| K/(K+1)."""
    import os

    from paper_2209_00315_gb300 import capi
    from ot_inputs import cube_config_densities

    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "gauss_cube8_oracle.npz"))
    n, K, r0, r1 = cube_config_densities("gauss_cube8")
    mesh = capi.Mesh(n, kind="cube")
    mu = float(g["mu"])
    _, _, _, norms = capi.ot_residual(mesh, K, mu, T(g["phi"]), T(g["rho"]), T(g["s"]), T(r0), T(r1))
    assert norms[3] < 1e-10
    c, dv = capi.ot_cost_dual(mesh, K, T(g["phi"]), T(g["rho"]), T(r0), T(r1))
    assert abs(c - float(g["cost"])) < 1e-13 * c
    gap = mu * K / (K + 1)
    assert abs((c - dv) - gap) < 1e-6 * gap
