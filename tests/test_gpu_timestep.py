"""Implicit Euler time stepping on the CUDA path (paper_1502_04070_gb300/timestep.py, C-ABI
stokes_euler_rhs) against the oracle's (oracle/timestep.py); Sec. 1: one step is the generalized
Stokes system with beta = 1/dt.

* the right-hand side of a step equals the oracle's load vector of f + u^n / dt;
* float64 and mixed-precision trajectories equal the oracle's exact steps to the solve tolerance;
* mixed precision on a larger level: every step reaches its tolerance (checked with the oracle's
  matrix) and the discrete energy identity of the implicit Euler method holds for f = 0, g = 0;
* warm starts: near a steady state, a step started from the previous time level needs fewer
  cycles than the same solve started from zero.
"""
import numpy as np
import pytest

from oracle import fem
from oracle import timestep as ts
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(7)


def _velocity(d, seed):
    fn, _ = workloads.random_nodal(d.mesh.level, seed)
    u, _ = d.from_vec(d.to_vec(fn, np.zeros((d.n + 1, d.n + 1))))
    return u


def _forcing(k, seed):
    f0, g0 = workloads.random_nodal(k, seed, with_g=True)
    return lambda n: (f0 * (1.0 + 0.1 * np.sin(n)), g0 * np.cos(0.3 * n))


def test_euler_rhs_matches_oracle(discs):
    from paper_1502_04070_gb300.timestep import ImplicitEuler
    k, dt = 4, 1e-3
    d = discs[k]
    te = ImplicitEuler(k + 1, dt, precision="fp64")
    try:
        u0 = _velocity(d, 11)
        fn, gn = workloads.random_nodal(k, 12, with_g=True)
        f, g = te.solver.euler_rhs(dev(u0), dev(fn), dev(gn))
        F = ts.euler_rhs(d, dt, u0, fn, gn)
        fo, go = d.from_vec(F)
        scale = np.abs(F).max()
        assert np.abs(host(f) - fo).max() <= 1e-13 * scale
        assert np.abs(host(g) - go).max() <= 1e-13 * scale
    finally:
        te.close()


_REFS = {}


def _reference(d, dt, u0, forcing, steps):
    """The oracle's exact steps (one sparse LU per step length), shared by both precisions."""
    if dt not in _REFS:
        _REFS[dt] = ts.implicit_euler(d, dt, u0, forcing, steps)
    return _REFS[dt]


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-8), ("mixed", 1e-10, 1e-6)])
@pytest.mark.parametrize("dt", [1e-2, 1e-4])
def test_trajectory_matches_oracle(discs, dt, precision, tol, bound):
    """Five steps at k = 5.  Bounds: the oracle's own multigrid stopped at a relative residual of
    1e-12 (1e-10) stays within 1e-10 (6.2e-10) of the exact steps here; the bounds leave a factor
    of 100 (1600) for rounding order."""
    from paper_1502_04070_gb300.timestep import ImplicitEuler
    k, steps = 5, 5
    d = discs[k]
    u0 = _velocity(d, 21)
    forcing = _forcing(k, 22)
    ref = _reference(d, dt, u0, forcing, steps)
    te = ImplicitEuler(k + 1, dt, precision=precision, tol=tol, max_cycles=200)
    try:
        u, p = dev(u0), te.solver.zeros_p()
        reps = te.run(u, p, lambda n: tuple(dev(a) for a in forcing(n)), steps)
        assert len(reps) == steps and all(r.converged for r in reps)
        # the last level; the earlier ones enter it through the warm starts and the right-hand sides
        x = d.to_vec(host(u), host(p))
        assert np.abs(x - ref[-1]).max() <= bound * np.abs(ref[-1]).max()
    finally:
        te.close()


def test_mixed_precision_steps_and_energy_identity(discs):
    """k = 6, f = 0, g = 0: every step solves the oracle's step system to its tolerance, the energy
    decays, and the identity ||u'||^2 - ||u||^2 + ||u' - u||^2 + 2 dt (K u', u') = 0 holds up to
    the solve: its defect is 2 dt ((r_p, p') - (u', r_u)) for the residual r, about 1e-14 of
    ||u||^2 at a relative residual of 1e-10 (measured with the oracle's multigrid)."""
    from paper_1502_04070_gb300.timestep import ImplicitEuler
    k, dt, steps, tol = 6, 1e-3, 4, 1e-10
    d = discs[k]
    u0 = _velocity(d, 31)
    zero = (np.zeros((2, 2 * d.n + 1, 2 * d.n + 1)), np.zeros((d.n + 1, d.n + 1)))
    S = d.system(1.0 / dt)
    te = ImplicitEuler(k + 1, dt, precision="mixed", tol=tol, max_cycles=200)
    try:
        u, p = dev(u0), te.solver.zeros_p()
        fz, gz = dev(zero[0]), dev(zero[1])
        prev = d.to_vec(u0, zero[1])
        for n in range(steps):
            u_prev_lat = host(u)
            te.step(u, p, fz, gz)
            x = d.to_vec(host(u), host(p))
            F = ts.euler_rhs(d, dt, u_prev_lat, *zero)
            assert np.linalg.norm(F - S @ x) <= 1.0001 * tol * np.linalg.norm(F)
            m1, m0, md, a1 = ts.energy_terms(d, prev[:d.nu], x[:d.nu])
            assert m1 < m0
            assert abs(m1 - m0 + md + 2 * dt * a1) <= 1e-6 * m0
            prev = x
    finally:
        te.close()


def test_warm_start_needs_fewer_cycles():
    """Constant data from u = 0, k = 6, dt = 1e-2: the solution approaches the steady state, so
    the step started from the previous level needs fewer cycles than the same solve from zero.
    The oracle's float64 multigrid takes 25, 15, 11, 10, 10, 9 cycles warm against 25 every step
    cold; the test asks for at most 0.7 of the cold total after the first step."""
    from paper_1502_04070_gb300.timestep import ImplicitEuler
    k, dt, steps = 6, 1e-2, 6
    f0, g0 = workloads.random_nodal(k, 41, with_g=True)
    te = ImplicitEuler(k + 1, dt, precision="mixed", tol=1e-8, max_cycles=200)
    try:
        u, p = te.solver.zeros_u(), te.solver.zeros_p()
        fn, gn = dev(f0), dev(g0)
        warm, cold = [], []
        for _ in range(steps):
            f, g = te.solver.euler_rhs(u, fn, gn)
            _, _, rep0 = te.solver.solve(f, g, tol=1e-8, max_cycles=200)       # from zero
            cold.append(rep0.cycles)
            warm.append(te.step(u, p, fn, gn).cycles)
        assert all(w <= c + 1 for w, c in zip(warm, cold)), (warm, cold)
        assert sum(warm[1:]) <= 0.7 * sum(cold[1:]), (warm, cold)
    finally:
        te.close()


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-8), ("mixed", 1e-10, 1e-6)])
def test_graph_run_matches_oracle_and_host_steps(discs, precision, tol, bound):
    """The five steps of the trajectory test (k = 5, dt = 1e-2) as one CUDA-graph launch
    (stokes_euler_run): the last level matches the oracle's exact steps within the same bounds,
    every step meets its tolerance in the true float64 residual, and each step takes the cycles of
    the same step driven from the host (within one: the graph stops on the true residual after every
    cycle, the host loop on the refinement's updated one, confirmed at the end)."""
    from paper_1502_04070_gb300.timestep import ImplicitEuler
    k, steps, dt = 5, 5, 1e-2
    d = discs[k]
    u0 = _velocity(d, 21)
    forcing = _forcing(k, 22)
    ref = _reference(d, dt, u0, forcing, steps)
    te = ImplicitEuler(k + 1, dt, precision=precision, tol=tol, max_cycles=200)
    try:
        data = [tuple(dev(a) for a in forcing(n)) for n in range(1, steps + 1)]
        u, p = dev(u0), te.solver.zeros_p()
        cyc, rel = te.run_graph(u, p, [a for a, _ in data], [b for _, b in data])
        assert len(cyc) == steps and all(r <= tol for r in rel), rel
        x = d.to_vec(host(u), host(p))
        assert np.abs(x - ref[-1]).max() <= bound * np.abs(ref[-1]).max()
        u2, p2 = dev(u0), te.solver.zeros_p()
        reps = [te.step(u2, p2, a, b) for a, b in data]
        assert all(abs(c - max(1, r.cycles)) <= 1 for c, r in zip(cyc, reps)), (cyc, [r.cycles for r in reps])
        # a second launch of the same graph from the same start gives the same trajectory
        u3, p3 = dev(u0), te.solver.zeros_p()
        cyc3, _ = te.run_graph(u3, p3, [a for a, _ in data], [b for _, b in data])
        assert cyc3 == cyc and float((u3 - u).abs().max()) == 0.0
    finally:
        te.close()


def test_batched_trajectories_match_single_runs(discs):
    """Three independent trajectories (k = 3, 4, 5 with dt = 1e-2, 1e-3, 1e-4), four steps each, in one
    launch (stokes_batch_euler_run): each equals its own single-trajectory graph run (the same kernels
    on the same data) and the k = 5 one the oracle's exact steps."""
    from paper_1502_04070_gb300.timestep import BatchImplicitEuler, ImplicitEuler
    ks, dts, steps = [3, 4, 5], [1e-2, 1e-3, 1e-4], 4
    datas, u0s = [], []
    for i, k in enumerate(ks):
        d = discs[k]
        u0s.append(_velocity(d, 51 + i))
        fo = _forcing(k, 61 + i)
        datas.append([tuple(dev(a) for a in fo(n)) for n in range(1, steps + 1)])
    be = BatchImplicitEuler([k + 1 for k in ks], dts, precision="fp64", tol=1e-12, max_cycles=200)
    try:
        us = [dev(u0) for u0 in u0s]
        ps = [torch_zeros_p(k) for k in ks]
        cyc, rel = be.run(us, ps, [[a for a, _ in dd] for dd in datas], [[b for _, b in dd] for dd in datas])
        assert all(r <= 1e-12 for row in rel for r in row)
        for i, k in enumerate(ks):
            te = ImplicitEuler(k + 1, dts[i], precision="fp64", tol=1e-12, max_cycles=200)
            try:
                u, p = dev(u0s[i]), te.solver.zeros_p()
                c1, _ = te.run_graph(u, p, [a for a, _ in datas[i]], [b for _, b in datas[i]])
                assert c1 == cyc[i]
                assert float((u - us[i]).abs().max()) <= 1e-14 * float(u.abs().max())
            finally:
                te.close()
        d = discs[5]
        ref = ts.implicit_euler(d, dts[2], u0s[2], _forcing(5, 63), steps)
        x = d.to_vec(host(us[2]), host(ps[2]))
        assert np.abs(x - ref[-1]).max() <= 1e-8 * np.abs(ref[-1]).max()
    finally:
        be.close()


def torch_zeros_p(k):
    import torch
    n = 2 ** (k + 1)
    return torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda")
