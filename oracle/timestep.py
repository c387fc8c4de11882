"""Implicit time stepping of the time-dependent Stokes problem, the application the generalized
Stokes system comes from (Sec. 1: beta is proportional to the inverse time step).

TEST INFRASTRUCTURE (part of the oracle package): only tests, the smoke check and the benchmark's
CPU baseline may import it.

    u_t - Laplace u + grad p = f,  div u = g,  u = 0 on the boundary,
discretized in time by the implicit Euler method with step dt:
    -Laplace u^{n+1} + beta u^{n+1} + grad p^{n+1} = f^{n+1} + beta u^n,  div u^{n+1} = g^{n+1},
    beta = 1/dt,
i.e. one generalized Stokes system (eq. stokes, Sec. 1) per step, whose discrete right-hand side
is the load vector of the nodal data f^{n+1} + beta u^n (the velocity load is linear in the
nodal values: (f_h + beta u^n, phi_i) = M_U f + beta M_U u^n).  Reading where the paper is silent:
unit viscosity (another viscosity is a rescaling of t, p and f by the caller) and the implicit
Euler scheme.  Every step is solved exactly (sparse LU of the bordered system, factorised once
per step length, zero-mean pressure as the border).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def euler_rhs(disc: fem.Discretization, dt, u_prev_lat, f_nodal, g_nodal):
    """Load vector of the step: F = ((f_h + u^n / dt, phi_i), (g_h - mean, psi_i))."""
    beta = 1.0 / dt
    w = np.asarray(f_nodal, np.float64) + beta * np.asarray(u_prev_lat, np.float64)
    return disc.load(w, g_nodal, project_g=True)


def implicit_euler(disc: fem.Discretization, dt, u0_lat, forcing, n_steps):
    """n_steps implicit Euler steps from the velocity u0 (lattice layout, zero on the boundary).
    forcing(n) -> (f_nodal, g_nodal) of step n = 1 .. n_steps.  Returns the list of unknown vectors
    x^1 .. x^n (velocity on the interior nodes, then pressure)."""
    solve = step_solver(disc, dt)
    u = np.asarray(u0_lat, np.float64)
    out = []
    for n in range(1, n_steps + 1):
        fn, gn = forcing(n)
        x = solve(euler_rhs(disc, dt, u, fn, gn))
        out.append(x)
        u, _ = disc.from_vec(x)
    return out


def step_solver(disc: fem.Discretization, dt):
    """Exact solve of the step's system [[K + M/dt, B^T], [B, 0]] x = F with the zero-mean pressure
    condition w^T p = 0 as a border row and column (w = M_P 1); the matrix is the same for every
    step, so it is factorised once (sparse LU)."""
    S = disc.system(1.0 / dt)
    w = np.concatenate([np.zeros(disc.nu), disc.w])
    Sb = sp.bmat([[S, sp.csr_matrix(w[:, None])], [sp.csr_matrix(w[None, :]), None]]).tocsc()
    lu = spla.splu(Sb)
    n = S.shape[0]
    return lambda F: lu.solve(np.concatenate([F, [0.0]]))[:n]


def energy_terms(disc: fem.Discretization, x_prev_u, x_u):
    """For velocity vectors (interior unknowns) u^n, u^{n+1}: the terms of the implicit Euler
    energy identity (f = 0, g = 0): ||u^{n+1}||_M^2, ||u^n||_M^2, ||u^{n+1} - u^n||_M^2 and
    (K u^{n+1}, u^{n+1}) with M, K the velocity mass and stiffness matrices."""
    ni = disc.ni
    M, K = disc.Mi, disc.Ki

    def quad(A, v):
        return v[:ni] @ (A @ v[:ni]) + v[ni:] @ (A @ v[ni:])

    return quad(M, x_u), quad(M, x_prev_u), quad(M, x_u - x_prev_u), quad(K, x_u)
