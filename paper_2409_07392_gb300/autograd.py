"""The Relax objective as a differentiable torch function.

``f^(z) = (1/s) sum_j v_j^T Sigma_z^{-1} H_p v_j`` (Hutchinson's estimate of
``Tr(Sigma_z^{-1} H_p)``, eqs. 4 and 11, with the probes of MD iteration ``t``).  The
backward kernel emits ``d f^/d z_i = -(1/s) sum_j u_j^T H_i y_j`` with ``U = Sigma_z^{-1} V``
and ``Y = Sigma_z^{-1} H_p V`` -- the exact derivative of ``f^`` for fixed probes.  With
``recompute=True`` the forward keeps nothing but its arguments and the backward re-runs the
probe solves.
"""
import torch

from .api import Problem


class FiralObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, problem: Problem, seed: int, t: int, s: int, tol: float, maxit: int,
                fixed_iters: int, recompute: bool):
        f, U, Y = problem.objective_fwd(z.detach(), seed, t, s, tol, maxit, fixed_iters,
                                        keep=not recompute)
        ctx.problem = problem
        ctx.args = (seed, t, s, tol, maxit, fixed_iters)
        if recompute:
            ctx.save_for_backward(z.detach())
            ctx.UY = None
        else:
            ctx.save_for_backward(z.detach())
            ctx.UY = (U, Y)
        return torch.tensor(f, dtype=torch.float64, device=z.device)

    @staticmethod
    def backward(ctx, grad_out):
        (z,) = ctx.saved_tensors
        seed, t, s, tol, maxit, fixed_iters = ctx.args
        U, Y = ctx.UY if ctx.UY is not None else (None, None)
        g = ctx.problem.objective_bwd(z, seed, t, s, U=U, Y=Y, grad_out=float(grad_out), tol=tol,
                                      maxit=maxit, fixed_iters=fixed_iters)
        return g.to(z.dtype), None, None, None, None, None, None, None, None


def firal_objective(z, problem: Problem, *, seed=1, t=0, s=10, tol=1e-6, maxit=500,
                    fixed_iters=0, recompute=False):
    """Differentiable f^(z) on a prepared problem (see module docstring)."""
    return FiralObjective.apply(z, problem, seed, t, s, tol, maxit, fixed_iters, recompute)
