"""Cost gradient (adjoint solve) on the GPU against the oracle (needs a GPU).

* ot_cost_grad at an oracle-converged state equals the oracle's transposed-
  Jacobian solve (both in the area gauge: gradients are defined up to a
  multiple of |c'|), to 1e-8 relative with a tight outer tolerance.
* the autograd wrapper returns the same gradient;
* 32x32 squares, K = 16: central differences of the GPU interior-point cost
  along 16 seeded mass-preserving directions (8 in rho_in, 8 in rho_f,
  h = 1e-6, both runs converged to the same mu with a 1e-12 Newton tolerance)
  agree with the adjoint gradient, and the gradient approaches the envelope
  form read off the dual potential at t = 0 and t = 1 like O(mu) (the gap
  shrinks >= 10x from duality gap 1e-4 to 1e-6);
* the 128x128, K = 32 workload: the gradient after a full mixed-precision
  solve is finite, area-gauged and within 5% of the envelope form.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint, ipm
from ot_inputs import config_densities, make_density, mass_preserving_directions, mixture_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tight(**kw):
    from paper_2209_00315_gb300 import capi

    base = dict(final_newton_tol=1e-12, final_eps_out=1e-12, fgmres_restart=60, fgmres_max_iter=1200)
    base.update(kw)
    return capi.default_options(**base)


@pytest.mark.parametrize("n,K", [(4, 4), (6, 3)])
def test_cost_grad_matches_oracle_adjoint(gpu_lib, n, K):
    from paper_2209_00315_gb300 import capi

    d = ipm.discretise(n, K)
    r0 = make_density(n, *mixture_params(3 * n + K, 2), 1e-2)
    r1 = make_density(n, *mixture_params(3 * n + K + 50, 2), 1e-2)
    res = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(gap_tol=1e-4, final_newton_tol=1e-13))
    g0, g1 = adjoint.cost_gradient(d, res.phi, res.rho, res.s, r0, r1)
    mesh = capi.Mesh(n)
    gin, gf = capi.ot_cost_grad(mesh, K, res.mu, T(res.phi), T(res.rho), T(res.s), T(r0), T(r1), options=tight())
    # the library returns the area-gauge representative itself (|c'| . grad = 0)
    for g in (gin, gf):
        gn = g.cpu().numpy()
        assert abs(d.t.coarse.area @ gn) < 1e-13 * np.linalg.norm(gn) * np.linalg.norm(d.t.coarse.area)
    assert rel(gin.cpu().numpy(), g0) < 1e-8
    assert rel(gf.cpu().numpy(), g1) < 1e-8


def test_autograd_wrapper_returns_the_adjoint_gradient(gpu_lib):
    from paper_2209_00315_gb300 import capi
    from paper_2209_00315_gb300.autograd import transport_cost

    n, K, r0, r1 = config_densities("gauss8")
    mesh = capi.Mesh(n)
    a = T(r0).requires_grad_(True)
    b = T(r1).requires_grad_(True)
    c = transport_cost(mesh, a, b, K, tol=1e-4, options=tight())
    ga, gb = torch.autograd.grad(3.0 * c, (a, b))
    res = capi.ot_ipm_solve(mesh, T(r0), T(r1), K, tol=1e-4, options=tight())
    assert abs(float(c) - res["cost"]) < 1e-12 * res["cost"]
    gin, gf = capi.ot_cost_grad(mesh, K, res["stats"]["mu"], res["phi"], res["rho"], res["s"], T(r0), T(r1),
                                options=tight())
    d = ipm.discretise(n, K)
    assert rel(ga, 3.0 * adjoint.area_gauge(d, gin.cpu().numpy())) < 1e-9
    assert rel(gb, 3.0 * adjoint.area_gauge(d, gf.cpu().numpy())) < 1e-9
    area = mesh.coarse_areas.to(DEV)
    assert abs(float(torch.dot(area, ga))) < 1e-12 * float(ga.norm())


@pytest.mark.slow
def test_cost_grad_central_differences_and_envelope_fd32(gpu_lib):
    """The differentiation check of the 128x128 workload, run at 32x32 squares, K = 16 (fd32 inputs)."""
    from paper_2209_00315_gb300 import capi

    n, K, r0, r1 = config_densities("fd32")
    d = ipm.discretise(n, K)
    mesh = capi.Mesh(n)
    opt = tight(precision="mixed")
    base = capi.ot_ipm_solve(mesh, T(r0), T(r1), K, options=opt)
    mu = base["stats"]["mu"]
    gin, gf = capi.ot_cost_grad(mesh, K, mu, base["phi"], base["rho"], base["s"], T(r0), T(r1), options=opt)
    g0 = adjoint.area_gauge(d, gin.cpu().numpy())
    g1 = adjoint.area_gauge(d, gf.cpu().numpy())
    # envelope form read off the GPU potential: the distance shrinks like mu
    # (two decades of mu between gap 1e-4 and 1e-6)
    e0, e1 = adjoint.envelope_gradient(d, base["phi"].cpu().numpy())
    far = capi.ot_ipm_solve(mesh, T(r0), T(r1), K, tol=1e-4, options=opt)
    fin, ff = capi.ot_cost_grad(mesh, K, far["stats"]["mu"], far["phi"], far["rho"], far["s"], T(r0), T(r1),
                                options=opt)
    f0, f1 = adjoint.envelope_gradient(d, far["phi"].cpu().numpy())
    near_err = max(rel(g0, e0), rel(g1, e1))
    far_err = max(rel(adjoint.area_gauge(d, fin.cpu().numpy()), f0), rel(adjoint.area_gauge(d, ff.cpu().numpy()), f1))
    assert near_err < far_err / 10 and near_err < 0.05, (near_err, far_err)
    # The cost is that of the unique barrier solution at mu: each perturbed
    # problem is solved at that mu directly, warm-started from the base point.
    dirs = mass_preserving_directions(n, 16, 8)
    h = 1e-6
    worst = 0.0
    warm = (base["rho"], base["phi"], base["s"])
    for i, v in enumerate(dirs):
        end = 0 if i < 8 else 1
        shift = lambda sgn: (T(r0 + sgn * h * v), T(r1)) if end == 0 else (T(r0), T(r1 + sgn * h * v))  # noqa
        cp = capi.ot_ipm_solve(mesh, *shift(+1), K, mu0=mu, options=opt, warm_start=warm)
        cm = capi.ot_ipm_solve(mesh, *shift(-1), K, mu0=mu, options=opt, warm_start=warm)
        assert cp["stats"]["stages"] == 1 and cp["stats"]["mu"] == mu and cm["stats"]["mu"] == mu
        fd = (cp["cost"] - cm["cost"]) / (2 * h)
        ad = float((g0 if end == 0 else g1) @ v)
        worst = max(worst, abs(fd - ad) / max(abs(fd), 1e-12))
    assert worst < 1e-4, worst


def test_cost_grad_at_the_128x128_workload(gpu_lib):
    """The differentiation workload itself: 128x128 squares (32768 coarse / 131072
    fine cells), K = 32, mixtures of seeds 4/5, mixed precision, solved to duality
    gap 1e-6 with the paper's tolerances.  The adjoint gradient is returned in the
    area gauge (zero sum), is finite, and lies within 5% of the envelope form
    -M'phi(0), M'phi(1) (with the (dt/4) R_E^T W (grad phi)^2 terms) read off the
    GPU potential, the distance that the fd32 check shows shrinking like mu."""
    from paper_2209_00315_gb300 import capi

    n, K, r0, r1 = config_densities("mix128")
    mesh = capi.Mesh(n)
    opt = capi.default_options(precision="mixed")
    res = capi.ot_ipm_solve(mesh, T(r0), T(r1), K, options=opt)
    st = res["stats"]
    assert st["stages"] == 10 and st["gap"] <= 1e-6
    gin, gf = capi.ot_cost_grad(mesh, K, st["mu"], res["phi"], res["rho"], res["s"], T(r0), T(r1), options=opt)
    g0, g1 = gin.cpu().numpy(), gf.cpu().numpy()
    assert np.isfinite(g0).all() and np.isfinite(g1).all()
    assert abs(g0.sum()) < 1e-10 * np.abs(g0).sum() and abs(g1.sum()) < 1e-10 * np.abs(g1).sum()
    d = ipm.discretise(n, K)
    e0, e1 = adjoint.envelope_gradient(d, res["phi"].cpu().numpy())
    err = max(rel(g0, e0), rel(g1, e1))
    print(f"\n128x128, K=32: adjoint gradient vs envelope form at gap 1e-6: {err:.2e}")
    assert err < 0.05, err
