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

A whole sequence of steps can also run as ONE CUDA-graph launch (stokes_euler_run: right-hand side,
warm-started device-side multigrid loop and step results per step, no host round trip), and
independent trajectories with their own step lengths and levels run concurrently in one launch
(BatchImplicitEuler, stokes_batch_euler_run).

This module only sequences library calls; every arithmetic step runs in the CUDA library.
"""
import ctypes

import torch

from . import _binding as B
from .solver import BatchSolver, Solver


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


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

    def run_graph(self, u, p, f_nodal, g_nodal):
        """len(f_nodal) steps in place as one graph launch; f_nodal[n], g_nodal[n] are the nodal data of
        time level n + 1 (the same tensor may repeat).  Returns (cycles per step, relative residual per
        step); raises if a step missed the tolerance."""
        S = self.solver
        n = len(f_nodal)
        if n < 1 or len(g_nodal) != n:
            raise ValueError("f_nodal and g_nodal must list the same positive number of steps")
        for t in list(f_nodal):
            S._chk(t, S.shape_u, "f_nodal")
        for t in list(g_nodal):
            S._chk(t, S.shape_p, "g_nodal")
        cyc = (ctypes.c_int * n)()
        rel = (ctypes.c_double * n)()
        st = S._lib.stokes_euler_run(S._h, S._chk(u, S.shape_u, "u"), S._chk(p, S.shape_p, "p"), _ptrs(f_nodal),
                                     _ptrs(g_nodal), n, self.tol, self.max_cycles, cyc, rel)
        B.check(st, "stokes_euler_run")
        return list(cyc), list(rel)

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


class BatchImplicitEuler:
    """Independent implicit Euler trajectories (instance i: level levels[i], step dts[i]) advanced
    together, each a chain of steps, all in one CUDA-graph launch."""

    def __init__(self, levels, dts, *, precision="mixed", tol=1e-8, max_cycles=100, **batch_kw):
        if any(not dt > 0.0 for dt in dts):
            raise ValueError("every dt must be positive")
        self.tol = float(tol)
        self.max_cycles = int(max_cycles)
        self.batch = BatchSolver(levels, [1.0 / dt for dt in dts], precision=precision, **batch_kw)

    def run(self, us, ps, f_nodal, g_nodal):
        """us, ps: per instance state tensors (in place); f_nodal[i][n], g_nodal[i][n]: nodal data of time
        level n + 1 of instance i (every instance the same number of steps).  Returns (cycles, relative
        residuals), each a list per instance of lists per step."""
        b = self.batch
        cnt = b.count
        steps = len(f_nodal[0])
        if len(us) != cnt or len(ps) != cnt or len(f_nodal) != cnt or len(g_nodal) != cnt or \
                any(len(f) != steps or len(g) != steps for f, g in zip(f_nodal, g_nodal)) or steps < 1:
            raise ValueError("one state and the same number of steps per instance")
        for i in range(cnt):
            su, sp = b.shapes(i)
            for t, sh in [(us[i], su), (ps[i], sp)] + [(t, su) for t in f_nodal[i]] + [(t, sp) for t in g_nodal[i]]:
                if t.dtype != torch.float64 or tuple(t.shape) != sh or not t.is_contiguous() or t.device != b.device:
                    raise ValueError("instance %d: expected contiguous float64 tensors of shape %s" % (i, sh))
        flat_f = [t for fi in f_nodal for t in fi]
        flat_g = [t for gi in g_nodal for t in gi]
        cyc = (ctypes.c_int * (cnt * steps))()
        rel = (ctypes.c_double * (cnt * steps))()
        st = b._lib.stokes_batch_euler_run(b._h, _ptrs(us), _ptrs(ps), _ptrs(flat_f), _ptrs(flat_g), steps, self.tol,
                                           self.max_cycles, cyc, rel)
        B.check(st, "stokes_batch_euler_run")
        return ([list(cyc[i * steps:(i + 1) * steps]) for i in range(cnt)],
                [list(rel[i * steps:(i + 1) * steps]) for i in range(cnt)])

    def close(self):
        self.batch.close()
