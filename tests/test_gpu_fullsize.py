"""Mixed precision at h = 1/2048 (k = 10, 37.7 M unknowns), beta = 1e4, manufactured solution
u = curl(sin^2(pi x) sin^2(pi y)), p = cos(pi x) cos(pi y): checks that hold at any size, since the
oracle cannot assemble this level in seconds.

* the mixed-precision solve reaches 1e-8 relative residual in float64, and so does the plain float64
  path; the two solutions agree to the size the residual bound allows;
* the nodal error against the analytic solution drops like h^2 or faster from k = 9 to k = 10
  (Taylor-Hood, Sec. 2; the discrete p approximates -p, see the weak form of Sec. 2);
* symmetry of the operator, <A x, y> = <x, A y>, through the float64 residual entry point;
* the Galerkin identity <I x_c, A_k I y_c> = <x_c, A_{k-1} y_c> through the transfer entry points.
"""
import math

import numpy as np
import pytest

from paper_1502_04070_gb300 import workloads

pytestmark = pytest.mark.gpu


def _nodal_errors(k, u, p):
    n, m2, m1 = workloads.sizes(k)
    t2 = np.arange(m2) / (2.0 * n)
    X, Y = np.meshgrid(t2, t2)
    ux, uy = workloads.exact_u(X, Y)
    t1 = np.arange(m1) / float(n)
    Xp, Yp = np.meshgrid(t1, t1)
    pe = -workloads.exact_p(Xp, Yp)
    uh = u.cpu().numpy()
    ph = p.cpu().numpy()
    eu = max(np.abs(uh[0] - ux).max(), np.abs(uh[1] - uy).max()) / np.abs(ux).max()
    ep = np.abs(ph - pe).max() / np.abs(pe).max()
    return eu, ep


def _solve(k, precision, tol=1e-8):
    import torch
    from paper_1502_04070_gb300.solver import Solver
    fn, gn = workloads.manufactured_nodal(k, 1e4)
    S = Solver(k + 1, 1e4, precision=precision)
    f, g = S.load_vectors(torch.from_numpy(fn).cuda(), torch.from_numpy(gn).cuda(), project_g=True)
    u, p, rep = S.solve(f, g, tol=tol, max_cycles=200)
    return S, f, g, u, p, rep


def test_h2048_mixed_and_fp64_manufactured():
    import torch
    S, f, g, u, p, rep = _solve(10, "mixed")
    assert rep.converged and rep.rel_residual <= 1e-8
    S64, _, _, u64, p64, rep64 = _solve(10, "fp64")
    assert rep64.converged and rep64.rel_residual <= 1e-8
    # the float64 residual entry point confirms the mixed result independently of the solve loop
    r = S64.residual_norm(u, p, f, g)
    nF = math.sqrt(float((f * f).sum() + (g * g).sum()))   # boundary entries of f are zero
    assert r <= 1.0001e-8 * nF
    du = float((u - u64).abs().max()) / float(u64.abs().max())
    assert du < 1e-3, du
    # discretisation error: both levels solved far below it (1e-10 relative residual)
    _, _, _, u10, p10, rep10 = _solve(10, "mixed", tol=1e-10)
    _, _, _, u9, p9, rep9 = _solve(9, "mixed", tol=1e-10)
    assert rep10.converged and rep9.converged
    eu10, ep10 = _nodal_errors(10, u10, p10)
    eu9, ep9 = _nodal_errors(9, u9, p9)
    assert eu10 < 0.3 * eu9 and ep10 < 0.3 * ep9, (eu9, eu10, ep9, ep10)


def test_h2048_operator_symmetry_and_galerkin_identity():
    import torch
    from paper_1502_04070_gb300.solver import Solver
    k, beta = 10, 1e4
    Sf = Solver(k + 1, beta)
    Sc = Solver(k, beta)
    x_u, x_p = [torch.from_numpy(a).cuda() for a in workloads.random_state(k, 1)]
    y_u, y_p = [torch.from_numpy(a).cuda() for a in workloads.random_state(k, 2)]
    zu, zp = Sf.zeros_u(), Sf.zeros_p()

    def apply(S, u, p):                      # A x = -(0 - A x)
        ru, rp = S.residual(u, p, torch.zeros_like(u), torch.zeros_like(p))
        return -ru, -rp

    ax_u, ax_p = apply(Sf, x_u, x_p)
    ay_u, ay_p = apply(Sf, y_u, y_p)
    lhs = float((ax_u * y_u).sum() + (ax_p * y_p).sum())
    rhs = float((x_u * ay_u).sum() + (x_p * ay_p).sum())
    scale = float((ax_u.abs() * y_u.abs()).sum() + (ax_p.abs() * y_p.abs()).sum())
    assert abs(lhs - rhs) <= 1e-12 * scale
    # Galerkin identity with coarse random states (k - 1)
    cx_u, cx_p = [torch.from_numpy(a).cuda() for a in workloads.random_state(k - 1, 3)]
    cy_u, cy_p = [torch.from_numpy(a).cuda() for a in workloads.random_state(k - 1, 4)]
    px_u, px_p = Sf.zeros_u(), Sf.zeros_p()
    py_u, py_p = Sf.zeros_u(), Sf.zeros_p()
    Sf.prolong_add(cx_u, cx_p, px_u, px_p)
    Sf.prolong_add(cy_u, cy_p, py_u, py_p)
    a_u, a_p = apply(Sf, py_u, py_p)
    fine = float((px_u * a_u).sum() + (px_p * a_p).sum())
    c_u, c_p = apply(Sc, cy_u, cy_p)
    coarse = float((cx_u * c_u).sum() + (cx_p * c_p).sum())
    scale = float((px_u.abs() * a_u.abs()).sum() + (px_p.abs() * a_p.abs()).sum())
    assert abs(fine - coarse) <= 1e-11 * scale, (fine, coarse)
