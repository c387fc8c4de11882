"""Adjoint multigrid gradients through torch.autograd (StokesSolve) against the oracle's adjoint
(direct solves) and against central finite differences of float64 solves."""
import numpy as np
import pytest

from oracle import adjoint, fem
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu


def _loss_grads(S, fn, gn, ut, beta, tol, max_cycles):
    import torch
    from paper_1502_04070_gb300.autograd import mass_half_norm2, stokes_solve
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    f = f.clone().requires_grad_(True)
    g = g.clone().requires_grad_(True)
    b = torch.tensor(beta, dtype=torch.float64, device="cuda", requires_grad=True)
    u, p = stokes_solve(f, g, b, S, tol=tol, max_cycles=max_cycles)
    L = mass_half_norm2(u - dev(ut), S)
    L.backward()
    return float(L), f.grad, g.grad, float(b.grad), f.detach(), g.detach()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_adjoint_matches_oracle(precision, tol):
    from paper_1502_04070_gb300.solver import Solver
    k, beta = 4, 30.0
    ds = fem.discretizations(k + 1)
    d = ds[-1]
    fn, gn = workloads.random_nodal(k, 11)
    ut, _ = workloads.random_nodal(k, 12)
    S = Solver(k + 1, beta, precision=precision)
    L, gf, gg, gb, f, g = _loss_grads(S, fn, gn, ut, beta, tol, 300)
    H = mg.Hierarchy(k + 1, beta, ds)
    F = d.load(fn, gn, project_g=True)
    utv = d.to_vec(ut, np.zeros((d.n + 1, d.n + 1)))[:d.nu]
    x, gF, gbo = adjoint.solve_and_gradients(H, F, lambda x: adjoint.loss_velocity_mass(d, x, utv)[1])
    Lo = adjoint.loss_velocity_mass(d, x, utv)[0]
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    got = d.to_vec(host(gf), host(gg))
    assert rel_err(got, gF) < (1e-8 if precision == "fp64" else 1e-6)
    assert abs(gb - gbo) <= (1e-8 if precision == "fp64" else 1e-6) * abs(gbo)


def test_adjoint_h1024_against_finite_differences():
    """h = 1/1024 (k = 9), beta = 1e3, L = 1/2 ||u - u_target||_M^2 with u_target uniform[-1,1]
    nodal (seed 5); mixed-precision forward and backward.  dL/df, dL/dg, dL/dbeta against central
    differences of float64 solves with a fixed number of cycles (the solve is then one fixed linear
    map of F, so the differences carry no stopping-rule noise), on 16 random directions in (f, g)
    plus beta.  Steps: L is exactly quadratic in F, so a central difference is exact for any step;
    the step is 1e-2 relative to ||F||, which keeps the float64 rounding noise of the solves
    (about 1e-9 relative at this size) below 1e-6 of the difference.  In beta, Richardson
    extrapolation of central differences with steps 1e-2 and 5e-3 relative."""
    import torch
    from paper_1502_04070_gb300.solver import Solver
    k, beta = 9, 1e3
    fn, gn = workloads.random_nodal(k, 5)
    ut, _ = workloads.random_nodal(k, 50)
    S = Solver(k + 1, beta, precision="mixed")
    L, gf, gg, gb, f, g = _loss_grads(S, fn, gn, ut, beta, 1e-9, 300)
    S64 = Solver(k + 1, beta)
    _, _, rep = S64.solve(f, g, tol=1e-11, max_cycles=300)
    ncyc = rep.cycles + 4

    def loss(ff, gg_, b):
        if S64.beta != b:
            S64.set_beta(b)
        u, p, _ = S64.solve(ff, gg_, tol=0.0, max_cycles=ncyc)
        e = u - dev(ut)
        return 0.5 * S64.mass_dot(e, e)

    rng = np.random.default_rng(17)
    nF = float(torch.sqrt((f * f).sum() + (g * g).sum()))
    errs = []
    for _ in range(16):
        du = dev(rng.standard_normal(f.shape))
        du[:, 0, :] = 0; du[:, -1, :] = 0; du[:, :, 0] = 0; du[:, :, -1] = 0
        dg = dev(rng.standard_normal(g.shape))
        S64.make_consistent(dg)
        scale = nF / float(torch.sqrt((du * du).sum() + (dg * dg).sum()))
        du, dg = du * scale, dg * scale
        h = 1e-2
        fd = (loss(f + h * du, g + h * dg, beta) - loss(f - h * du, g - h * dg, beta)) / (2 * h)
        an = float((gf * du).sum() + (gg * dg).sum())
        errs.append(abs(fd - an) / max(abs(fd), 1e-300))
    assert max(errs) < 1e-5, errs
    cd = lambda hb: (loss(f, g, beta + hb) - loss(f, g, beta - hb)) / (2 * hb)
    hb = 1e-2 * beta
    fdb = (4.0 * cd(hb / 2) - cd(hb)) / 3.0
    assert abs(fdb - gb) <= 1e-5 * abs(fdb), (fdb, gb)
