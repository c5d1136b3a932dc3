"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

Operators are compared element by element on seeded random states; Newton
directions against the oracle's sparse-LU solution; full interior-point
solves on small meshes (several thread blocks with ragged tails) in FP64 and
mixed precision.  Tolerances: 1e-8 relative in the cost and 1e-6 relative L2
in rho and phi for solves (the accuracy target of the solver); operators and
directions are FP64 computations of the same sums in another order, compared
at 1e-12.
"""
import numpy as np
import pytest
import torch

from oracle import ipm
from ot_inputs import config_densities, make_density

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def random_state(d, seed):
    rng = np.random.default_rng(seed)
    phi = 0.3 * rng.standard_normal((d.K + 1) * d.N)
    rho = rng.uniform(0.5, 2, d.K * d.Nc)
    s = rng.uniform(0.5, 2, d.K * d.Nc)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    rho = ipm.renormalise(d, rho, r0)
    return phi, rho, s, r0, r1


SIZES = [(1, 1), (2, 3), (5, 2), (6, 3), (10, 2)]


@pytest.fixture(scope="module")
def cases(gpu_lib):
    from paper_2209_00315_gb300 import capi

    out = []
    for n, K in SIZES:
        d = ipm.discretise(n, K)
        out.append((n, K, d, capi.Mesh(n), random_state(d, 100 * n + K)))
    return out


def test_residual_matches_oracle(cases):
    from paper_2209_00315_gb300 import capi

    for n, K, d, mesh, (phi, rho, s, r0, r1) in cases:
        F = ipm.residual(d, phi, rho, s, r0, r1, 0.37)
        G = capi.ot_residual(mesh, K, 0.37, T(phi), T(rho), T(s), T(r0), T(r1))
        for a, b in zip(G[:3], F):
            assert rel(a, b) < 1e-13, (n, K)
        assert abs(G[3][3] - ipm.residual_norm(F)) < 1e-12 * ipm.residual_norm(F)


def test_projected_kkt_operator_matches_oracle(cases):
    from paper_2209_00315_gb300 import capi

    for n, K, d, mesh, (phi, rho, s, r0, r1) in cases:
        Kp = d.projected_kkt(phi, rho, s, r0, r1)
        x = np.random.default_rng(n + K).standard_normal(Kp.shape[0])
        y = capi.ot_kkt_apply(mesh, K, T(phi), T(rho), T(s), T(r0), T(r1), T(x))
        assert rel(y, Kp @ x) < 1e-13, (n, K)


def test_schur_operator_matches_oracle(cases):
    from paper_2209_00315_gb300 import capi

    for n, K, d, mesh, (phi, rho, s, r0, r1) in cases:
        S = d.schur_bb(phi, rho, s)
        z = np.random.default_rng(7 + n).standard_normal(S.shape[0])
        out = capi.ot_schur_apply(mesh, K, T(phi), T(rho), T(s), T(z))
        assert rel(out, S @ z) < 1e-13, (n, K)


@pytest.mark.parametrize("n,K,phi_kind", [(2, 2, "random"), (4, 3, "random"), (32, 2, "smooth")])
def test_bb_application_matches_exact_oracle(gpu_lib, n, K, phi_kind):
    """One application of the BB preconditioner (Sec. 4.3.3) in FP64 with the inner
    Schur GMRES driven to 1e-13 and 60 V-cycles per slice Laplacian, against the
    oracle's application with sparse-LU solves.  x is compared after removing each
    slice's mean, the constant that the singular slice Laplacians leave free.  At
    n = 32 (8192 cells per slice) the finest Laplacian level is swept in device
    memory and the coarser ones in shared memory; below, all in shared memory.
    The large case takes a smooth phi: cell-wise random potentials have gradients
    growing as 1/h, which makes the Schur block indefinite from n = 8 on (real
    parts of its eigenvalues down to -89 at n = 16) and no longer a state the
    interior-point method visits."""
    from paper_2209_00315_gb300 import capi
    from oracle import operators as ops

    d = ipm.discretise(n, K)
    phi, rho, s, r0, r1 = random_state(d, 7 * n + K)
    if phi_kind == "smooth":
        c = d.t.fine.centre
        wave = np.sin(2 * np.pi * c[:, 0]) * np.cos(np.pi * c[:, 1])
        phi = np.concatenate([0.1 * wave * (k / K) for k in range(K + 1)])
    else:
        phi = 0.1 * phi
    Np = (K + 1) * d.N
    v = np.random.default_rng(5).standard_normal(Np + K * d.Nc)
    x, y = ops.bb_apply_exact(d, phi, rho, s, r0, r1, v)
    opt = capi.default_options(precision="fp64", eps_schur=1e-13, schur_max_iter=400, lap_cycles=60)
    out = capi.ot_bb_apply(capi.Mesh(n), K, T(phi), T(rho), T(s), T(r0), T(r1), T(v), options=opt)
    out = out.cpu().numpy()
    gx = out[:Np].reshape(K + 1, d.N)
    gx = (gx - gx.mean(axis=1, keepdims=True)).ravel()
    assert rel(gx, x) < 1e-10, (n, K)
    assert rel(out[Np:], y) < 1e-10, (n, K)


def test_cost_and_dual_match_oracle(cases):
    from paper_2209_00315_gb300 import capi

    for n, K, d, mesh, (phi, rho, s, r0, r1) in cases:
        c, dv = capi.ot_cost_dual(mesh, K, T(phi), T(rho), T(r0), T(r1))
        assert abs(c - ipm.cost(d, phi, rho, r0, r1)) < 1e-13 * abs(c)
        assert abs(dv - ipm.dual_value(d, phi, r0, r1)) < 1e-12 * max(1.0, abs(dv))


@pytest.mark.parametrize("n,K", [(1, 1), (1, 2), (2, 1), (2, 2), (2, 3), (4, 4)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_newton_direction_matches_dense_lu(gpu_lib, n, K, precision):
    """FGMRES + BB with a tight tolerance reproduces the exact Newton direction (LU)."""
    from paper_2209_00315_gb300 import capi

    d = ipm.discretise(n, K)
    phi, rho, s, r0, r1 = random_state(d, 11 * n + K)
    phi *= 0.03  # a smooth-ish potential: BB assumes grad phi varies slowly (Sec. 4.3.2)
    mu = 0.05
    mesh = capi.Mesh(n)
    opt = capi.default_options(eps_out=1e-13, fgmres_restart=60, fgmres_max_iter=600, precision=precision)
    dphi, drho, ds, st = capi.ot_newton_solve(mesh, K, mu, T(phi), T(rho), T(s), T(r0), T(r1), options=opt)
    ophi, orho, os_, _ = ipm.newton_direction(d, phi, rho, s, r0, r1, mu)
    assert rel(dphi, ophi) < 1e-10 and rel(drho, orho) < 1e-10 and rel(ds, os_) < 1e-10
    assert st["fgmres_iters"] < 600


def _ipm_pair(n, K, r0, r1, precision="fp64"):
    from paper_2209_00315_gb300 import capi

    mesh = capi.Mesh(n)
    opt = capi.default_options(final_newton_tol=1e-11, final_eps_out=1e-10, precision=precision)
    res = capi.ot_ipm_solve(mesh, T(r0), T(r1), K, options=opt)
    d = ipm.discretise(n, K)
    ref = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(final_newton_tol=1e-11))
    return d, res, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ipm_matches_oracle_gaussians_8x8(gpu_lib, precision):
    """Gaussians sigma = 0.1 at (0.3,0.3) -> (0.7,0.7), 8x8 squares, K = 8, floor 1e-3, gap 1e-6."""
    n, K, r0, r1 = config_densities("gauss8")
    d, res, ref = _ipm_pair(n, K, r0, r1, precision)
    assert abs(res["cost"] - ref.cost) < 1e-8 * ref.cost
    assert rel(res["rho"], ref.rho) < 1e-6
    assert rel(res["phi"], ref.phi) < 1e-6
    st = res["stats"]
    assert st["stages"] == 10 and abs(st["gap"] - ref.mu * K / (K + 1)) < 1e-20
    assert abs((st["cost"] - st["dual"]) - st["gap"]) < 1e-6 * st["gap"]


@pytest.mark.parametrize("n,K,seed", [(6, 3, 1), (10, 5, 2)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ipm_matches_oracle_mixtures(gpu_lib, n, K, seed, precision):
    from ot_inputs import mixture_params

    r0 = make_density(n, *mixture_params(seed, 3), 1e-4)
    r1 = make_density(n, *mixture_params(seed + 50, 3), 1e-4)
    d, res, ref = _ipm_pair(n, K, r0, r1, precision)
    assert abs(res["cost"] - ref.cost) < 1e-8 * ref.cost
    assert rel(res["rho"], ref.rho) < 1e-6 and rel(res["phi"], ref.phi) < 1e-6
    assert float(res["rho"].min()) > 0 and float(res["s"].min()) > 0


def test_uniform_densities_exact(gpu_lib):
    """Degenerate case rho_in = rho_f = const: exact solution, one Newton step per stage."""
    from paper_2209_00315_gb300 import capi

    n, K = 4, 3
    r0 = np.ones(2 * n * n)
    mesh = capi.Mesh(n)
    res = capi.ot_ipm_solve(mesh, T(r0), T(r0), K, options=capi.default_options(final_newton_tol=1e-12))
    st = res["stats"]
    assert all(v == 1 for v in st["stage_newton"])
    assert torch.allclose(res["rho"], torch.ones_like(res["rho"]), atol=1e-13, rtol=0)
    assert abs(res["cost"]) < 1e-20


def test_host_memspace_path(gpu_lib):
    """Numpy inputs go through host pointers (copies inside the library) and give the same answer."""
    from paper_2209_00315_gb300 import capi

    n, K = 4, 4
    r0 = make_density(n, [(0.3, 0.3)], [0.1], [1.0], 1e-3)
    r1 = make_density(n, [(0.7, 0.7)], [0.1], [1.0], 1e-3)
    mesh = capi.Mesh(n)
    a = capi.ot_ipm_solve(mesh, r0, r1, K)
    b = capi.ot_ipm_solve(mesh, T(r0), T(r1), K)
    assert not a["rho"].is_cuda
    assert abs(a["cost"] - b["cost"]) < 1e-12 * b["cost"]
    assert rel(a["rho"], b["rho"].cpu().numpy()) < 1e-12


def test_errors_are_returned_not_raised_on_device(gpu_lib):
    from paper_2209_00315_gb300 import capi

    n, K = 2, 2
    mesh = capi.Mesh(n)
    good = np.ones(2 * n * n)
    with pytest.raises(capi.OTError) as e:
        capi.ot_ipm_solve(mesh, T(good), T(2 * good), K)
    assert e.value.code == 2
    bad = good.copy()
    bad[0] = -1.0
    with pytest.raises(capi.OTError) as e:
        capi.ot_ipm_solve(mesh, T(bad), T(good), K)
    assert e.value.code == 3
    nan = good.copy()
    nan[1] = np.nan
    with pytest.raises(capi.OTError) as e:
        capi.ot_ipm_solve(mesh, T(nan), T(good), K)
    assert e.value.code == 6
    # Newton cap of 1 at mu0 = 1 from the interpolated start: not converged
    with pytest.raises(capi.OTError) as e:
        r0 = make_density(n, [(0.3, 0.3)], [0.1], [1.0], 1e-3)
        r1 = make_density(n, [(0.7, 0.7)], [0.1], [1.0], 1e-3)
        capi.ot_ipm_solve(mesh, T(r0), T(r1), K, options=capi.default_options(max_newton=1))
    assert e.value.code == 4
    # the context is still usable afterwards
    res = capi.ot_ipm_solve(mesh, T(good), T(good), K)
    assert abs(res["cost"]) < 1e-20


@pytest.mark.slow
def test_full_size_mix64_against_oracle_properties(gpu_lib):
    """The benchmark workload (64x64 squares, K = 32, mixed precision, default
    options, as bench.py runs it) checked with the oracle at full size, through
    properties the oracle evaluates directly: its residual at the GPU solution
    meets the final Newton tolerance, its cost and dual value reproduce the
    GPU's, the duality gap is mu |Omega| K/(K+1), masses are conserved slice by
    slice, and rho, s > 0."""
    from paper_2209_00315_gb300 import capi

    n, K, r0, r1 = config_densities("mix64")
    mesh = capi.Mesh(n)
    res = capi.ot_ipm_solve(mesh, T(r0), T(r1), K, options=capi.default_options(precision="mixed"))
    st = res["stats"]
    d = ipm.discretise(n, K)
    phi, rho, s = (res[k].cpu().numpy() for k in ("phi", "rho", "s"))
    mu = st["mu"]
    F = ipm.residual(d, phi, rho, s, r0, r1, mu)
    fn = ipm.residual_norm(F)
    # the oracle's ||F|| at the returned point is the GPU's own final ||F||, which met R6
    assert abs(fn - st["final_residual"]) <= 1e-6 * st["final_residual"] + 1e-13, (fn, st["final_residual"])
    assert fn < 1e-6
    c = ipm.cost(d, phi, rho, r0, r1)
    dv = ipm.dual_value(d, phi, r0, r1)
    assert abs(c - res["cost"]) < 1e-12 * c
    assert abs(dv - st["dual"]) < 1e-10 * max(1.0, abs(dv))
    # C - D - mu |Omega| K/(K+1) = dt (phi.F_phi - rho.F_rho + |c'|.F_s) at any point (summation
    # by parts; pinned on the oracle): the gap error is what the final residual implies, bounded by
    # Cauchy-Schwarz with the norms of the returned point and of its residual
    gap = mu * d.area_total * K / (K + 1)
    Fphi, Frho, Fs = F
    cw = np.tile(d.t.coarse.area, K)
    implied = d.dt * (phi @ Fphi - rho @ Frho + cw @ Fs)
    assert abs((c - dv) - gap - implied) < 1e-9 * (abs(c) + abs(dv)), (c - dv - gap, implied)
    bound = d.dt * (np.linalg.norm(phi) * np.linalg.norm(Fphi) + np.linalg.norm(rho) * np.linalg.norm(Frho)
                    + np.linalg.norm(cw) * np.linalg.norm(Fs))
    assert abs((c - dv) - gap) <= bound, (c - dv, gap, bound)
    mass = d.rho_slices(rho) @ d.t.coarse.area
    assert np.abs(mass - d.t.coarse.area @ r0).max() < 1e-12
    assert rho.min() > 0 and s.min() > 0


@pytest.mark.parametrize("n,K", [(4, 1), (4, 40), (2, 130)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ipm_matches_oracle_time_slice_extremes(gpu_lib, n, K, precision):
    """Edge cases of the time dimension: a single density slice (K = 1), two PCR
    lines per lane (32 < K <= 64: the K-slice line solves span two registers per
    lane), and K > 128, where the line smoothers fall back to one Thomas sweep
    per thread and no level is fused."""
    from ot_inputs import mixture_params

    r0 = make_density(n, *mixture_params(900 + n, 2), 1e-3)
    r1 = make_density(n, *mixture_params(950 + K, 2), 1e-3)
    d, res, ref = _ipm_pair(n, K, r0, r1, precision)
    assert abs(res["cost"] - ref.cost) < 1e-8 * ref.cost
    assert rel(res["rho"], ref.rho) < 1e-6 and rel(res["phi"], ref.phi) < 1e-6


@pytest.mark.parametrize("n,K", [(1, 2), (4, 4), (8, 6)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ipm_matches_oracle_disjoint_supports(gpu_lib, n, K, precision):
    """Densities with zeros: rho_in lives on the left half, rho_f on the right
    half (allowed: only rho_in + rho_f > 0 is required); n = 1 is the smallest
    mesh (two coarse triangles, one multigrid level on the space-time side)."""
    from ot_inputs import coarse_triangles

    cx = coarse_triangles(n)[:, :, 0].mean(1)
    d = ipm.discretise(n, K)
    area = d.t.coarse.area
    r0 = np.where(cx < 0.5, 1.0, 0.0)
    r1 = np.where(cx >= 0.5, 1.0, 0.0)
    r0, r1 = r0 / (area @ r0), r1 / (area @ r1)
    d, res, ref = _ipm_pair(n, K, r0, r1, precision)
    assert abs(res["cost"] - ref.cost) < 1e-8 * ref.cost
    assert rel(res["rho"], ref.rho) < 1e-6 and rel(res["phi"], ref.phi) < 1e-6
    assert float(res["rho"].min()) > 0
