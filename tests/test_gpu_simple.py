"""The SIMPLE preconditioner and the SIMPLE/BB hybrid on the GPU against the oracle (needs a GPU).

SIMPLE (Sec. 4.2) on the projected system with A^ = Diag(A): x1 = A^-1 c,
y = S^-1 (d - P B x1) with S^ = -(P C P^T + P B A^-1 B^T P^T), x = x1 -
A^-1 B^T P^T y.  With its inner Schur GMRES driven to 1e-13 the GPU
application must equal the oracle's (`operators.simple_apply_exact`, a
bordered sparse-LU solve) to FP64 rounding.  Full interior-point solves with
SIMPLE throughout, and with the hybrid that switches from BB to SIMPLE below a
barrier parameter (the paper's proposal for small mu), must reach the oracle's
solution at the parity tolerances (1e-8 cost, 1e-6 rho and phi): the
preconditioner changes the iteration counts, not the answer.
"""
import numpy as np
import pytest
import torch

from oracle import ipm
from ot_inputs import make_density, mixture_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def random_state(d, seed, smooth_phi=False):
    rng = np.random.default_rng(seed)
    if smooth_phi:
        c = d.t.fine.centre
        wave = np.sin(2 * np.pi * c[:, 0]) * np.cos(np.pi * c[:, 1])
        phi = np.concatenate([0.1 * wave * (k / d.K) for k in range(d.K + 1)])
    else:
        phi = 0.03 * rng.standard_normal((d.K + 1) * d.N)
    rho = rng.uniform(0.5, 2, d.K * d.Nc)
    s = rng.uniform(0.5, 2, d.K * d.Nc)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    rho = ipm.renormalise(d, rho, r0)
    return phi, rho, s, r0, r1


@pytest.mark.parametrize("n,K,precision,smooth", [(1, 1, "fp64", False), (2, 3, "fp64", False),
                                                  (4, 3, "mixed", False), (5, 6, "fp64", False),
                                                  (16, 4, "fp64", True)])
def test_simple_application_matches_exact_oracle(gpu_lib, n, K, precision, smooth):
    """One SIMPLE application with the inner GMRES to 1e-13 against the oracle's
    exact application; both precisions run SIMPLE in FP64.  Sizes span one to
    many thread blocks (n = 16: 2048 fine cells per slice) and the K = 1 edge
    case, where the time lines have a single slice."""
    from paper_2209_00315_gb300 import capi
    from oracle import operators as ops

    d = ipm.discretise(n, K)
    phi, rho, s, r0, r1 = random_state(d, 31 * n + K, smooth)
    Np = (K + 1) * d.N
    rng = np.random.default_rng(9 + n)
    v = rng.standard_normal(Np + K * d.Nc)
    v[Np:] = d.P_block() @ v[Np:]                # d in the range of P, as the projected system's rows are
    x, y = ops.simple_apply_exact(d, phi, rho, s, r0, r1, v)
    opt = capi.default_options(precision=precision, eps_schur=1e-13, schur_max_iter=400)
    out = capi.ot_simple_apply(capi.Mesh(n), K, T(phi), T(rho), T(s), T(r0), T(r1), T(v), options=opt)
    out = out.cpu().numpy()
    assert rel(out[:Np], x) < 1e-10, (n, K)
    assert rel(out[Np:], y) < 1e-10, (n, K)
    # y in the range of P^T: zero area-weighted slice sums
    assert np.abs(out[Np:].reshape(K, d.Nc).sum(axis=1)).max() < 1e-12 * max(np.abs(y).max(), 1.0) * d.Nc


def test_simple_inner_solve_is_preconditioned_by_the_time_lines(gpu_lib):
    """Where the potential has no spatial gradient, the time-line part is all of
    SIMPLE's Schur complement: its preconditioner is then exact and the inner
    GMRES converges in one iteration."""
    from paper_2209_00315_gb300 import capi
    from oracle import operators as ops

    n, K = 8, 6
    d = ipm.discretise(n, K)
    _, rho, s, r0, r1 = random_state(d, 77)
    phi = np.repeat(np.linspace(-0.2, 0.3, K + 1), d.N)      # constant in space: grad phi = 0
    Np = (K + 1) * d.N
    v = np.random.default_rng(3).standard_normal(Np + K * d.Nc)
    v[Np:] = d.P_block() @ v[Np:]
    x, y = ops.simple_apply_exact(d, phi, rho, s, r0, r1, v)
    opt = capi.default_options(precision="fp64", eps_schur=1e-12, schur_max_iter=1)
    out = capi.ot_simple_apply(capi.Mesh(n), K, T(phi), T(rho), T(s), T(r0), T(r1), T(v), options=opt)
    out = out.cpu().numpy()
    assert rel(out[:Np], x) < 1e-11 and rel(out[Np:], y) < 1e-11


def _solve(n, K, r0, r1, precision, **kw):
    from paper_2209_00315_gb300 import capi

    opt = capi.default_options(precision=precision, final_newton_tol=1e-11, final_eps_out=1e-10, **kw)
    return capi.ot_ipm_solve(capi.Mesh(n), T(r0), T(r1), K, options=opt)


@pytest.mark.parametrize("precond,simple_mu", [("simple", 1e-5), ("hybrid", 1e-3)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ipm_with_simple_matches_oracle(gpu_lib, precond, simple_mu, precision):
    """4x4 squares, K = 16 (time finer than space, the regime where SIMPLE pays),
    3-Gaussian mixtures of seeds 2/3, floor 1e-4: SIMPLE throughout, and the
    hybrid switching to SIMPLE for the stages with mu < 1e-3 (the last five of
    ten), against the oracle's exact-Newton solution."""
    n, K = 4, 16
    r0 = make_density(n, *mixture_params(2, 3), 1e-4)
    r1 = make_density(n, *mixture_params(3, 3), 1e-4)
    d = ipm.discretise(n, K)
    ref = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(final_newton_tol=1e-11))
    res = _solve(n, K, r0, r1, precision, precond=precond, simple_mu=simple_mu)
    assert abs(res["cost"] - ref.cost) < 1e-8 * ref.cost
    assert rel(res["rho"], ref.rho) < 1e-6 and rel(res["phi"], ref.phi) < 1e-6
    st = res["stats"]
    assert st["stages"] == 10 and abs(st["mu"] - ref.mu) < 1e-20
