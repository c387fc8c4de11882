"""Implicit time stepping of the time-dependent Stokes problem on top of the multigrid solver.

Sec. 1: the generalized Stokes system is the system of one step of an implicit time
discretization, beta proportional to the inverse step length.  For
    u_t - Laplace u + grad p = f,  div u = g,  u = 0 on the boundary   (unit viscosity)
the implicit Euler method with step dt solves, per step,
    -Laplace u^{n+1} + beta u^{n+1} + grad p^{n+1} = f^{n+1} + beta u^n,  div u^{n+1} = g^{n+1},
with beta = 1/dt: the library forms the right-hand side (stokes_euler_rhs) and solves it by
multigrid from the previous time level (a warm start; stokes_solve with the iterate given), all
on the device.  Another viscosity nu is the same problem with beta = 1/(nu dt), data f/nu and
pressure p/nu, which the caller applies.

This module only sequences library calls; every arithmetic step runs in the CUDA library.
"""
from .solver import Solver


class ImplicitEuler:
    """Implicit Euler steps of fixed length dt: one generalized Stokes solve (beta = 1/dt) each."""

    def __init__(self, levels: int, dt: float, *, precision="mixed", tol=1e-8, max_cycles=100, **solver_kw):
        if not dt > 0.0:
            raise ValueError("dt must be positive")
        self.dt = float(dt)
        self.tol = float(tol)
        self.max_cycles = int(max_cycles)
        self.solver = Solver(levels, 1.0 / self.dt, precision=precision, **solver_kw)
        self.reports = []

    @property
    def shape_u(self):
        return self.solver.shape_u

    @property
    def shape_p(self):
        return self.solver.shape_p

    def step(self, u, p, f_nodal, g_nodal):
        """Advances (u, p) by one step in place, from u^n to u^{n+1}; f_nodal, g_nodal are the nodal
        data of time level n+1.  The solve starts from (u^n, p^n).  Returns the solve report and
        raises if the solve did not reach the tolerance."""
        f, g = self.solver.euler_rhs(u, f_nodal, g_nodal)
        _, _, rep = self.solver.solve(f, g, tol=self.tol, max_cycles=self.max_cycles, u=u, p=p,
                                      raise_on_fail=True)
        self.reports.append(rep)
        return rep

    def run(self, u, p, forcing, n_steps):
        """n_steps steps in place; forcing(n) -> (f_nodal, g_nodal) of time level n = 1 .. n_steps.
        Returns the reports of the steps."""
        out = []
        for n in range(1, n_steps + 1):
            fn, gn = forcing(n)
            out.append(self.step(u, p, fn, gn))
        return out

    def close(self):
        self.solver.close()
