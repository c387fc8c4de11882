"""Gradients of a loss through the discrete generalized Stokes solve (adjoint method).

The discrete solution x = (u, p) of eq. gen:bil:mv with the zero-mean pressure condition is the
first block of the bordered system  [[S(beta), w], [w^T, 0]] [x; mu] = [F; 0],  w = (0, M_P 1),
S(beta) = [[K + beta M_U, B^T], [B, 0]].  S is symmetric (Sec. 2), hence so is the bordered matrix,
and for a loss L(x):
    lambda = first block of the bordered solve with right-hand side [dL/dx; 0]
    dL/dF  = lambda                         (dL/df = lambda_u, dL/dg = lambda_p)
    dL/dbeta = -lambda^T (dS/dbeta) x = -lambda_u^T M_U u.
lambda_p is the representative with w^T lambda_p = 0 that the bordered solve produces; any constant
shift of it gives the same derivative in every admissible direction (sum(dg) = 0).
"""
import numpy as np

from . import multigrid as mg


def solve_and_gradients(H: mg.Hierarchy, F, dL_dx_fn):
    """Direct solve of the finest level, then the adjoint solve.  dL_dx_fn(x) -> dL/dx.
    Returns x, dL/dF, dL/dbeta."""
    l = len(H.levels) - 1
    d = H.discs[l]
    x = H.direct(F)
    lam = mg.direct_solve(H.levels[l].S, d, dL_dx_fn(x))
    u, lam_u = x[:d.nu], lam[:d.nu]
    dbeta = -lam_u @ (d.mass_u() @ u)
    return x, lam, dbeta


def loss_velocity_mass(d, x, u_target):
    """L = 1/2 (u - u_t)^T M_U (u - u_t) and its gradient with respect to x."""
    e = x[:d.nu] - u_target
    Me = d.mass_u() @ e
    grad = np.zeros_like(x)
    grad[:d.nu] = Me
    return 0.5 * e @ Me, grad
