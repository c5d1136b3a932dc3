"""Gradient of the discrete cost with respect to the end densities (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

At a point u = (phi, rho, s) where G(u; r0, r1) = (F_phi; F_rho; F_s - mu) = 0
(Sec. 2.3-2.4), the barrier solution is a function u(r0, r1) of the end
densities r0 = rho^0 and r1 = rho^{K+1}.  The cost C(phi, rho; r0, r1) of
reading R15 then has the total derivative (adjoint method)

    dC/dr = dC/dr|_u - (dG/dr)^T lam,     J^T lam = (dC/du)^T,

with J = dG/du the Jacobian of Eq. (newton-linsys).  The pieces, written from
the formulas of F and C:

  C = dt sum_k 1/2 W rho~^k (grad phi^k)^2,  rho~^k = R_E (r_k + r_{k-1})/2 over the
      extended list r_0 = r0, r_1..r_K = rho, r_{K+1} = r1 (paper k = 1..K+1), so
      dC/dphi^k = dt grad^T (W rho~^k grad phi^k),
      dC/dr_j   = dt/4 R_E^T W [(grad phi^j)^2 + (grad phi^{j+1})^2]   (terms that exist);
  G depends on r0 only through F_phi^1 and on r1 only through F_phi^{K+1}:
      dF_phi^1/dr0       =  M J/dt - 1/2 div Diag(grad phi^1) R_E,
      dF_phi^{K+1}/dr1   = -M J/dt - 1/2 div Diag(grad phi^{K+1}) R_E.

J^T has the constant potential (1, 0, 0) as null vector, and dC/dphi is
orthogonal to it (C is invariant under phi -> phi + const), so the system is
consistent; one potential unknown is grounded as in ipm.newton_direction.  The
free constant of lam moves both gradients by a multiple of the coarse areas
|c'| (J^T M 1 = |c'|), which no mass-preserving direction sees: gradients are
compared after removing their component along |c'| (``area_gauge``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .ipm import jacobian
from .operators import Discretisation


def cost_partials(d: Discretisation, phi, rho, rho0, rho1):
    """(dC/dphi, dC/drho, dC/dr0, dC/dr1) at fixed u (reading R15)."""
    P = d.phi_slices(phi)
    rt = d.rho_tilde(rho, rho0, rho1)
    g = [d.grad @ P[k] for k in range(d.K + 1)]
    dphi = np.concatenate([d.dt * (d.grad.T @ (d.W * rt[k] * g[k])) for k in range(d.K + 1)])
    e = [0.25 * d.dt * (d.RE.T @ (d.W * g[k] * g[k])) for k in range(d.K + 1)]
    drho = np.concatenate([e[j - 1] + e[j] for j in range(1, d.K + 1)])   # r_j sits in rho~^j and rho~^{j+1}
    return dphi, drho, e[0], e[d.K]


def end_density_jacobians(d: Discretisation, phi):
    """dF_phi^1/dr0 and dF_phi^{K+1}/dr1 (N x N' each)."""
    P = d.phi_slices(phi)
    MJ = (d.M @ d.J).tocsr()
    flux = lambda k: (-0.5 * (d.div @ (sp_diag(d.grad @ P[k]) @ d.RE))).tocsr()  # noqa: E731
    return (MJ / d.dt + flux(0)).tocsr(), (-MJ / d.dt + flux(d.K)).tocsr()


def sp_diag(v):
    return sp.diags(np.asarray(v))


def adjoint_state(d: Discretisation, phi, rho, s, rho0, rho1):
    """lam = (lam_phi, lam_rho, lam_s) solving J^T lam = (dC/du)^T, first potential grounded."""
    dphi, drho, _, _ = cost_partials(d, phi, rho, rho0, rho1)
    Np, Nr = (d.K + 1) * d.N, d.K * d.Nc
    rhs = np.concatenate([dphi, drho, np.zeros(Nr)])
    JT = jacobian(d, phi, rho, s, rho0, rho1).T.tocsc()
    sub = JT[1:, :][:, 1:].tocsc()
    lam = np.zeros(JT.shape[0])
    lam[1:] = spla.splu(sub).solve(rhs[1:])
    return lam[:Np], lam[Np:Np + Nr], lam[Np + Nr:]


def cost_gradient(d: Discretisation, phi, rho, s, rho0, rho1):
    """(dC/dr0, dC/dr1), each N', in the area gauge."""
    _, _, c0, c1 = cost_partials(d, phi, rho, rho0, rho1)
    lam_phi, _, _ = adjoint_state(d, phi, rho, s, rho0, rho1)
    L = d.phi_slices(lam_phi)
    D0, D1 = end_density_jacobians(d, phi)
    return area_gauge(d, c0 - D0.T @ L[0]), area_gauge(d, c1 - D1.T @ L[d.K])


def area_gauge(d: Discretisation, g):
    """g minus its least-squares component along the coarse areas |c'|."""
    a = d.t.coarse.area
    return np.asarray(g) - (np.dot(a, g) / np.dot(a, a)) * a


def envelope_gradient(d: Discretisation, phi):
    """Partial derivatives of the dual value D (reading R15) in r0 and r1 at fixed phi:
        dD/dr0 = -J^T M phi^1     - dt/4 R_E^T W (grad phi^1)^2,
        dD/dr1 =  J^T M phi^{K+1} - dt/4 R_E^T W (grad phi^{K+1})^2.
    C - D is the constant mu |Omega| K/(K+1) along the barrier solutions, and D
    becomes stationary in phi as mu -> 0, so these approach dC/dr0, dC/dr1 at
    rate O(mu) (envelope argument); returned in the area gauge."""
    P = d.phi_slices(phi)
    MJt = (d.M @ d.J).T.tocsr()
    g1, gK = d.grad @ P[0], d.grad @ P[-1]
    q0 = 0.25 * d.dt * (d.RE.T @ (d.W * g1 * g1))
    q1 = 0.25 * d.dt * (d.RE.T @ (d.W * gK * gK))
    return area_gauge(d, -(MJt @ P[0]) - q0), area_gauge(d, (MJt @ P[-1]) - q1)
