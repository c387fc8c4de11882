"""Pins of the oracle's implicit Euler time stepping (oracle/timestep.py), the application of
Sec. 1 (beta = 1/dt):

* the discrete energy identity of the implicit Euler method for f = 0, g = 0:
  ||u^{n+1}||_M^2 - ||u^n||_M^2 + ||u^{n+1} - u^n||_M^2 + 2 dt (K u^{n+1}, u^{n+1}) = 0
  (test the step with u^{n+1}; the pressure term drops out because B u^{n+1} = 0);
* the steady Stokes solution (beta = 0) is a fixed point of the step for constant data, and the
  iteration converges to it from zero;
* started from a discrete Stokes eigenfunction (K v + B^T q = lambda M v, B v = 0, from a dense
  generalized eigensolver), the steps are u^n = (1 + dt lambda)^(-n) v.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fem
from oracle import multigrid as mg
from oracle import timestep as ts
from paper_1502_04070_gb300 import workloads


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(4)


def _random_velocity(d, seed):
    fn, _ = workloads.random_nodal(d.mesh.level, seed)
    x = d.to_vec(fn, np.zeros((d.n + 1, d.n + 1)))     # interior values only
    u, _ = d.from_vec(x)
    return u


@pytest.mark.parametrize("dt", [1e-1, 1e-3])
def test_energy_identity(discs, dt):
    d = discs[3]
    u0 = _random_velocity(d, 3)
    zero = (np.zeros((2, 2 * d.n + 1, 2 * d.n + 1)), np.zeros((d.n + 1, d.n + 1)))
    xs = ts.implicit_euler(d, dt, u0, lambda n: zero, 4)
    prev = d.to_vec(u0, np.zeros((d.n + 1, d.n + 1)))[:d.nu]
    for x in xs:
        u = x[:d.nu]
        m1, m0, md, a1 = ts.energy_terms(d, prev, u)
        assert abs(m1 - m0 + md + 2 * dt * a1) <= 1e-11 * m0
        assert m1 < m0                                   # the energy decays
        prev = u


def test_steady_solution_is_fixed_point(discs):
    d = discs[3]
    fn, gn = workloads.random_nodal(3, 8, with_g=True)
    F = d.load(fn, gn, project_g=True)
    xs_ = mg.direct_solve(d.system(0.0), d, F)
    us, ps = d.from_vec(xs_)
    x1 = ts.implicit_euler(d, 0.05, us, lambda n: (fn, gn), 1)[0]
    assert np.abs(x1 - xs_).max() <= 1e-11 * np.abs(xs_).max()
    x = ts.implicit_euler(d, 0.1, np.zeros_like(us), lambda n: (fn, gn), 40)[-1]
    assert np.abs(x - xs_).max() <= 1e-9 * np.abs(xs_).max()


@pytest.mark.parametrize("dt", [1e-2, 1e-3])
def test_stokes_eigenfunction_decays_by_closed_form(discs, dt):
    d = discs[1]
    nu, nv = d.nu, d.nv
    K = sp.block_diag([d.Ki, d.Ki]).toarray()
    M = sp.block_diag([d.Mi, d.Mi]).toarray()
    B = d.Bi.toarray()
    w = d.w
    n = nu + nv + 1
    A = np.zeros((n, n))
    A[:nu, :nu] = K
    A[:nu, nu:nu + nv] = B.T
    A[nu:nu + nv, :nu] = B
    A[nu:nu + nv, -1] = w
    A[-1, nu:nu + nv] = w
    Bm = np.zeros((n, n))
    Bm[:nu, :nu] = M
    lam, V = sla.eig(A, Bm)
    ok = np.isfinite(lam) & (np.abs(lam.imag) < 1e-8 * np.abs(lam)) & (lam.real > 1e-8)
    j = np.flatnonzero(ok)[np.argmin(lam.real[ok])]
    lmb = lam.real[j]
    v = V[:nu, j].real
    v /= np.abs(v).max()
    assert np.abs(B @ v).max() < 1e-10                     # divergence-free
    u0, _ = d.from_vec(np.concatenate([v, np.zeros(nv)]))
    zero = (np.zeros((2, 2 * d.n + 1, 2 * d.n + 1)), np.zeros((d.n + 1, d.n + 1)))
    xs = ts.implicit_euler(d, dt, u0, lambda m: zero, 3)
    for m, x in enumerate(xs, start=1):
        assert np.abs(x[:nu] - (1 + dt * lmb) ** -m * v).max() <= 1e-10
