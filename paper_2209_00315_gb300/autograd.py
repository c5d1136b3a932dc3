"""Differentiable transport cost.

``transport_cost(mesh, rho_in, rho_f, K)`` runs the interior-point solve
(Sec. 3) to the requested duality gap on the GPU and returns the discrete cost
C (the kinetic energy of the discrete flow: dt sum_k 1/2 sum_e |e||w| rho~ (grad phi)^2)
as a 0-dim tensor.  Its backward pass is one adjoint solve at the converged
point: the transposed Jacobian, which after eliminating the slack is the same
symmetric saddle operator as the Newton systems, solved by the same FGMRES +
BB preconditioner (``ot_cost_grad``).  It returns dC/d rho_in and dC/d rho_f
times the incoming gradient.

The masses of rho_in and rho_f must stay equal, so only mass-preserving
perturbations are admissible and each gradient is defined up to a multiple of
the coarse cell areas |c'|; ot_cost_grad returns the representative with that
component removed (the area gauge).
"""
import torch

from . import capi


class TransportCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho_in, rho_f, mesh, K, mu0, tol, options):
        r0 = rho_in.detach().to(torch.float64).contiguous()
        r1 = rho_f.detach().to(torch.float64).contiguous()
        res = capi.ot_ipm_solve(mesh, r0, r1, K, mu0=mu0, tol=tol, options=options)
        ctx.mesh, ctx.K, ctx.options, ctx.mu = mesh, K, options, res["stats"]["mu"]
        ctx.save_for_backward(r0, r1, res["phi"], res["rho"], res["s"])
        return torch.tensor(res["cost"], dtype=torch.float64, device=rho_in.device)

    @staticmethod
    def backward(ctx, grad_out):
        r0, r1, phi, rho, s = ctx.saved_tensors
        gin, gf = capi.ot_cost_grad(ctx.mesh, ctx.K, ctx.mu, phi, rho, s, r0, r1, options=ctx.options)
        return gin * grad_out, gf * grad_out, None, None, None, None, None


def transport_cost(mesh, rho_in, rho_f, K: int, mu0: float = 1.0, tol: float = 1e-6, options=None):
    """Discrete optimal-transport cost between rho_in and rho_f (CUDA tensors of
    N' cell averages, equal masses), differentiable in both densities."""
    if not (isinstance(rho_in, torch.Tensor) and rho_in.is_cuda and isinstance(rho_f, torch.Tensor) and rho_f.is_cuda):
        raise ValueError("transport_cost takes CUDA tensors")
    return TransportCost.apply(rho_in, rho_f, mesh, K, mu0, tol, options)
