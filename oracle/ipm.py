"""Residual, Jacobian, exact Newton directions and the interior-point loop (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 2.3-3 of the paper:
  F_phi^k = -M J (rho^k - rho^{k-1})/dt - div(R_E((rho^k + rho^{k-1})/2) * grad phi^k),  k = 1..K+1
  F_rho^k = J^T M (phi^{k+1} - phi^k)/dt + 1/4 R_T((grad phi^k)^2 + (grad phi^{k+1})^2) + M' s^k   (R3)
  F_s^k   = rho^k * s^k,   relaxed to F_s - mu = 0 by the log barrier (Eq. l2-discrete)
and each Newton step solves the Jacobian system (Eq. newton-linsys) exactly by
sparse LU, with the potential's free constant (Remark kernel) fixed by
sum(M dphi) = 0 after grounding one potential unknown.

Readings taken where the paper is silent, ambiguous or inconsistent:
  R4  the barrier weighs cell i of the density mesh by |c'_i|.
  R6  Newton stops at ||(F_phi; F_rho; F_s - mu)||_2 <= tol * max(1, ||F at stage start||).
  R7  mu_{l+1} = mu_l / 5 from mu_0; stop after the first stage whose gap
      mu |Omega| K/(K+1) is <= the requested tolerance.
  R8  initial point: rho^k = (1 - t_k) rho^0 + t_k rho^{K+1}, phi = 0, s = mu_0 / rho.
  R9  step length alpha = min(1, tau min_{d<0}(-x/d)) over rho and s, tau = 0.99;
      after each update every rho^k is rescaled to the mass of rho^0 (Remark zero-mean).
  R15 cost  C = dt sum_k 1/2 sum_e |e||w| rho~^k_e (grad phi^k)_e^2, and dual value
      D = phi^{K+1}.M J rho^{K+1} - phi^1.M J rho^0
          - dt/4 [(R_E rho^0).W (grad phi^1)^2 + (R_E rho^{K+1}).W (grad phi^{K+1})^2].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import one_level_cube, two_level_square
from .operators import Discretisation


def discretise(n: int, K: int) -> Discretisation:
    return Discretisation(two_level_square(n), K)


def discretise_cube(n: int, K: int) -> Discretisation:
    """The 3D Cartesian variant (the paper's test 4): n^3 cubes, J = I."""
    return Discretisation(one_level_cube(n), K)


# ------------------------------------------------------------------ residual
def residual(d: Discretisation, phi, rho, s, rho0, rho1, mu: float):
    """(F_phi, F_rho, F_s - mu), each flattened slice-major."""
    K, dt = d.K, d.dt
    P = d.phi_slices(phi)
    R = d.rho_ext(rho, rho0, rho1)
    S = d.rho_slices(s)
    rt = d.rho_tilde(rho, rho0, rho1)
    Fphi = np.empty((K + 1, d.N))
    for k in range(K + 1):                       # k here is the paper's k-1
        Fphi[k] = -(d.M @ (d.J @ (R[k + 1] - R[k]))) / dt - d.div @ (rt[k] * (d.grad @ P[k]))
    Frho = np.empty((K, d.Nc))
    JtM = d.J.T @ d.M
    for k in range(K):
        g0, g1 = d.grad @ P[k], d.grad @ P[k + 1]
        Frho[k] = JtM @ (P[k + 1] - P[k]) / dt + 0.25 * (d.RT @ (g0 ** 2 + g1 ** 2)) + d.Mc @ S[k]
    Fs = R[1:-1] * S - mu
    return Fphi.ravel(), Frho.ravel(), Fs.ravel()


def residual_norm(F) -> float:
    return float(np.sqrt(sum(float(np.dot(f, f)) for f in F)))


# ------------------------------------------------------------------ Jacobian
def dFphi_drho(d: Discretisation, phi) -> sp.csr_matrix:
    """Derivative of F_phi with respect to rho, written from the formula of F_phi."""
    K, dt = d.K, d.dt
    P = d.phi_slices(phi)
    MJ = (d.M @ d.J).tocsr()
    blocks = [[None] * K for _ in range(K + 1)]
    for j in range(K + 1):           # F_phi slice j (paper's j+1) depends on rho^{j+1}, rho^j
        Dg = (-d.div @ sp.diags(d.grad @ P[j]) @ d.RE * 0.5).tocsr()
        if j <= K - 1:   # rho^{j+1} (paper index) is unknown slice j
            blocks[j][j] = -MJ / dt + Dg
        if j >= 1:       # rho^{j} (paper index) is unknown slice j-1
            blocks[j][j - 1] = MJ / dt + Dg
    for j in range(K + 1):
        for k in range(K):
            if blocks[j][k] is None:
                blocks[j][k] = sp.csr_matrix((d.N, d.Nc))
    return sp.bmat(blocks).tocsr()


def jacobian(d: Discretisation, phi, rho, s, rho0, rho1) -> sp.csr_matrix:
    """The 3x3 block Jacobian of (F_phi; F_rho; F_s - mu), Eq. (newton-linsys)."""
    A = d.A_block(rho, rho0, rho1)
    B = d.B_block(phi)
    Mc = d.Mc_block()
    Z = lambda r, c: sp.csr_matrix((r, c))  # noqa: E731
    Np, Nr = (d.K + 1) * d.N, d.K * d.Nc
    return sp.bmat([
        [A, dFphi_drho(d, phi), Z(Np, Nr)],
        [B, Z(Nr, Nr), Mc],
        [Z(Nr, Np), sp.diags(np.asarray(s)), sp.diags(np.asarray(rho))],
    ]).tocsr()


def newton_direction(d: Discretisation, phi, rho, s, rho0, rho1, mu: float):
    """Exact solution of Eq. (newton-linsys) with sum(M dphi) = 0.

    The Jacobian is singular with kernel (1, 0, 0) (Remark kernel), and
    (1, 0, 0) is also its left null vector (A 1 = 0 and B 1 = 0).  The first
    unknown of dphi is grounded and the first potential equation dropped,
    which leaves a nonsingular sparse system; the free constant is then fixed
    by sum(M dphi) = 0.  The dropped equation holds automatically when the
    masses of rho^0 and rho^{K+1} agree; its residual is returned.
    """
    F = residual(d, phi, rho, s, rho0, rho1, mu)
    rhs = -np.concatenate(F)
    Jm = jacobian(d, phi, rho, s, rho0, rho1).tocsc()
    sub = Jm[1:, :][:, 1:].tocsc()
    sol = np.zeros(Jm.shape[0])
    sol[1:] = spla.splu(sub).solve(rhs[1:])
    dropped = float((Jm[0, :] @ sol)[0] - rhs[0])
    Np, Nr = (d.K + 1) * d.N, d.K * d.Nc
    w = np.tile(d.t.fine.area, d.K + 1)
    sol[:Np] -= np.dot(w, sol[:Np]) / w.sum()
    return sol[:Np], sol[Np:Np + Nr], sol[Np + Nr:], dropped


# ------------------------------------------------------------------ cost
def cost(d: Discretisation, phi, rho, rho0, rho1) -> float:
    """Discrete kinetic energy C (reading R15)."""
    P = d.phi_slices(phi)
    rt = d.rho_tilde(rho, rho0, rho1)
    total = 0.0
    for k in range(d.K + 1):
        g = d.grad @ P[k]
        total += 0.5 * float(np.dot(d.W * rt[k], g * g))
    return d.dt * total


def dual_value(d: Discretisation, phi, rho0, rho1) -> float:
    """Dual objective D (reading R15); C - D = mu |Omega| K/(K+1) at a solution."""
    P = d.phi_slices(phi)
    g1, gK = d.grad @ P[0], d.grad @ P[-1]
    MJ = d.M @ d.J
    term = float(P[-1] @ (MJ @ rho1)) - float(P[0] @ (MJ @ rho0))
    corr = float((d.RE @ rho0) @ (d.W * g1 * g1)) + float((d.RE @ rho1) @ (d.W * gK * gK))
    return term - 0.25 * d.dt * corr


def phi_gauge(d: Discretisation, phi) -> np.ndarray:
    """phi minus its M-weighted space-time mean (reading R11)."""
    w = np.tile(d.t.fine.area, d.K + 1)
    return phi - np.dot(w, phi) / w.sum()


# ------------------------------------------------------------------ IPM
@dataclass
class IPMOptions:
    mu0: float = 1.0
    mu_factor: float = 0.2
    gap_tol: float = 1e-6
    newton_tol: float = 1e-6
    final_newton_tol: float | None = None   # tighter tolerance for the last stage
    tau: float = 0.99
    max_newton: int = 60


@dataclass
class IPMResult:
    phi: np.ndarray
    rho: np.ndarray
    s: np.ndarray
    cost: float
    dual: float
    mu: float
    stages: list = field(default_factory=list)   # (mu, newton steps, final ||F||)
    newton_steps: int = 0


def initial_point(d: Discretisation, rho0, rho1, mu0: float):
    """Reading R8."""
    t = np.arange(1, d.K + 1)[:, None] * d.dt
    rho = ((1.0 - t) * rho0[None, :] + t * rho1[None, :]).ravel()
    phi = np.zeros((d.K + 1) * d.N)
    s = mu0 / rho
    return phi, rho, s


def step_length(x, dx, tau: float) -> float:
    """Fraction to the boundary (reading R9)."""
    neg = dx < 0
    if not np.any(neg):
        return 1.0
    return float(min(1.0, tau * np.min(-x[neg] / dx[neg])))


def renormalise(d: Discretisation, rho, rho0):
    """Rescale each rho^k to the mass of rho^0 (Remark zero-mean)."""
    R = d.rho_slices(rho).copy()
    area = d.t.coarse.area
    target = float(area @ rho0)
    R *= (target / (R @ area))[:, None]
    return R.ravel()


def stage_count(K: int, opt: IPMOptions, area_total: float = 1.0) -> int:
    """Number of mu stages until mu |Omega| K/(K+1) <= gap_tol (reading R7)."""
    mu, count = opt.mu0, 1
    while mu * area_total * K / (K + 1) > opt.gap_tol:
        mu *= opt.mu_factor
        count += 1
    return count


def ipm_solve(d: Discretisation, rho0, rho1, opt: IPMOptions | None = None, start=None) -> IPMResult:
    """Interior-point continuation in mu with exact Newton steps (Sec. 2.4, 3)."""
    opt = opt or IPMOptions()
    rho0 = np.asarray(rho0, dtype=np.float64)
    rho1 = np.asarray(rho1, dtype=np.float64)
    phi, rho, s = start if start is not None else initial_point(d, rho0, rho1, opt.mu0)
    n_stage = stage_count(d.K, opt, d.area_total)
    mu = opt.mu0
    res = IPMResult(phi, rho, s, 0.0, 0.0, mu)
    for stage in range(n_stage):
        F = residual(d, phi, rho, s, rho0, rho1, mu)
        f0 = residual_norm(F)
        last = stage == n_stage - 1
        tol = opt.final_newton_tol if (last and opt.final_newton_tol is not None) else opt.newton_tol
        tol = tol * max(1.0, f0)
        steps = 0
        fn = f0
        while fn > tol:
            if steps >= opt.max_newton:
                raise RuntimeError(f"Newton did not converge at mu={mu:g} (||F||={fn:.3e})")
            dphi, drho, ds, _ = newton_direction(d, phi, rho, s, rho0, rho1, mu)
            alpha = min(step_length(rho, drho, opt.tau), step_length(s, ds, opt.tau))
            phi = phi + alpha * dphi
            rho = renormalise(d, rho + alpha * drho, rho0)
            s = s + alpha * ds
            F = residual(d, phi, rho, s, rho0, rho1, mu)
            fn = residual_norm(F)
            steps += 1
        res.stages.append((mu, steps, fn))
        res.newton_steps += steps
        if stage < n_stage - 1:
            mu *= opt.mu_factor
    res.phi, res.rho, res.s, res.mu = phi, rho, s, mu
    res.cost = cost(d, phi, rho, rho0, rho1)
    res.dual = dual_value(d, phi, rho0, rho1)
    return res
