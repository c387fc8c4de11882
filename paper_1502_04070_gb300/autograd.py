"""Differentiable generalized Stokes solves: torch.autograd.Function with an adjoint multigrid backward.

Forward:  x = (u, p) solves  A(beta) x = F,  F = (f, g) load vectors, with int p = 0 (eq. gen:bil:mv;
          the zero-mean condition of Sec. 1 is the border of the system).
Backward: A(beta) is symmetric (Sec. 2), so the adjoint system is the forward one.  For incoming
          gradients (du, dp) the library solves A lam = (du, dp - (1^T dp) w), w = M_P 1 (the
          border makes the right-hand side consistent), with the same multigrid, and returns
              dL/df = lam_u,   dL/dg = lam_p,   dL/dbeta = -lam_u^T M_U u.
          lam_p carries the solver's zero-mean representative; every admissible direction of g
          (sum 0) sees the same derivative for any constant shift of it.
Nothing per level is stored between forward and backward: the backward pass re-runs the solver's
setup for beta (diagonals, coarse factorisation) if the solver was used for another beta meanwhile.
All arithmetic runs in the CUDA library; this module only routes tensors.
"""
import torch

from .solver import Solver


class StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, g, beta, solver: Solver, tol: float, max_cycles: int):
        b = float(beta)
        if solver.beta != b:
            solver.set_beta(b)
        u, p, rep = solver.solve(f.detach().contiguous(), g.detach().contiguous(), tol=tol,
                                 max_cycles=max_cycles, raise_on_fail=True)
        ctx.solver, ctx.tol, ctx.max_cycles, ctx.beta = solver, tol, max_cycles, b
        ctx.save_for_backward(u)
        return u, p

    @staticmethod
    def backward(ctx, du, dp):
        (u,) = ctx.saved_tensors
        S = ctx.solver
        if S.beta != ctx.beta:
            S.set_beta(ctx.beta)
        du = S.zeros_u() if du is None else du.detach().contiguous().clone()
        dp = S.zeros_p() if dp is None else dp.detach().contiguous().clone()
        S.make_consistent(dp)
        lam_u, lam_p, rep = S.solve(du, dp, tol=ctx.tol, max_cycles=ctx.max_cycles, raise_on_fail=True)
        dbeta = -S.mass_dot(lam_u, u)
        grad_beta = torch.tensor(dbeta, dtype=torch.float64, device=u.device)
        return lam_u, lam_p, grad_beta, None, None, None


def stokes_solve(f, g, beta, solver: Solver, tol: float = 1e-10, max_cycles: int = 200):
    """Differentiable (u, p) = A(beta)^{-1} (f, g); beta may be a float or a 0-d float64 tensor."""
    if not torch.is_tensor(beta):
        beta = torch.tensor(float(beta), dtype=torch.float64, device=f.device)
    return StokesSolve.apply(f, g, beta, solver, tol, max_cycles)


class MassInner(torch.autograd.Function):
    """1/2 a^T M_U a for a velocity array a with zero boundary entries (half the squared L2 norm of
    the P2 function), differentiable."""

    @staticmethod
    def forward(ctx, a, solver: Solver):
        ctx.solver = solver
        ctx.save_for_backward(a)
        return torch.tensor(0.5 * solver.mass_dot(a.detach().contiguous(), a.detach().contiguous()),
                            dtype=torch.float64, device=a.device)

    @staticmethod
    def backward(ctx, gout):
        (a,) = ctx.saved_tensors
        return gout * ctx.solver.mass_apply(a.detach().contiguous()), None


def mass_half_norm2(a, solver: Solver):
    return MassInner.apply(a, solver)
