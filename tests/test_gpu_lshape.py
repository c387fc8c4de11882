"""The L-shaped domain on the CUDA path (stokes_params.domain = STOKES_L_SHAPE: the square's lattice
with the closed upper-right quadrant masked; Sec. 1: the method applies to non-convex domains)
against the oracle's L (oracle/lshape.py: the kept triangles assembled on their own), element by
element, at L-levels j = 1..5 (square levels 2..6, N = 8..128 squares per side):

* the residual F - S x of eq. gen:bil:mv (1e-12, relative to the largest entry);
* one Uzawa smoothing step (Sec. 4) with the L's diagonals Ahat, Shat (1e-12);
* whole V and W cycles with the exact solve on the L's level 0 and the zero-mean pressure over the
  L (1e-10), and solves against the oracle's sparse direct solution;
* float32 cycles inside float64 refinement (STOKES_MIXED): the first step against one oracle cycle
  (1e-5) and solves against the direct solution (1e-8).
Entries outside the L are zero in every result.
"""
import numpy as np
import pytest

from oracle import lshape
from oracle import multigrid as mg
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu

JMAX = 5


@pytest.fixture(scope="module")
def ds():
    return lshape.discretizations(JMAX + 1)


def _masked_state(d, seed):
    """A random (u, p) and (f, g) on the L's unknowns, zero elsewhere, as lattice arrays."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, d.ndof)
    F = rng.uniform(-1, 1, d.ndof)
    F[d.nu:] -= F[d.nu:].mean()          # sum of g = 0: orthogonal to the constant pressure (solvable)
    u, p = d.from_vec(x)
    f, g = d.from_vec(F)
    return u, p, f, g, x, F


def _solver(j, beta, **kw):
    from paper_1502_04070_gb300.solver import Solver
    return Solver(j + 2, beta, domain="lshape", coarse_level=1, **kw)


def _outside_is_zero(d, u, p):
    xi = d.from_vec(d.to_vec(u, p))
    return np.abs(u - xi[0]).max() == 0.0 and np.abs(p - xi[1]).max() == 0.0


@pytest.mark.parametrize("j", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("beta", [0.0, 1e4])
def test_residual(ds, j, beta):
    d = ds[j]
    u, p, f, g, x, F = _masked_state(d, 10 + j)
    S = _solver(j, beta)
    ru, rp = S.residual(dev(u), dev(p), dev(f), dev(g))
    got_u, got_p = host(ru), host(rp)
    assert _outside_is_zero(d, got_u, got_p)
    ref = F - d.system(beta) @ x
    assert rel_err(d.to_vec(got_u, got_p), ref) < 1e-12
    S.close()


@pytest.mark.parametrize("j", [1, 3, 5])
@pytest.mark.parametrize("beta", [1.0, 1e6])
def test_uzawa_step(ds, j, beta):
    d = ds[j]
    u, p, f, g, x, F = _masked_state(d, 20 + j)
    lvl = mg.Level(d, beta)
    ref = mg.Hierarchy.uzawa_step(None, lvl, x, F, mg.Params())
    S = _solver(j, beta)
    tu, tp = dev(u), dev(p)
    S.smooth(tu, tp, dev(f), dev(g), 1)
    got_u, got_p = host(tu), host(tp)
    assert _outside_is_zero(d, got_u, got_p)
    assert rel_err(d.to_vec(got_u, got_p), ref) < 1e-12
    S.close()


@pytest.mark.parametrize("j", [1, 2, 4, 5])
@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("beta", [1.0, 1e6])
def test_cycle(ds, j, gamma, beta):
    d = ds[j]
    H = mg.Hierarchy(j + 1, beta, ds[:j + 1])
    u, p, f, g, x, F = _masked_state(d, 30 + j)
    prm = mg.Params(gamma=gamma)
    S = _solver(j, beta, gamma=gamma)
    tu, tp, tf, tg = dev(u), dev(p), dev(f), dev(g)
    for _ in range(2):
        x = H.project_mean(j, H.cycle(j, x, F, prm))
        S.cycle(tu, tp, tf, tg)
    got_u, got_p = host(tu), host(tp)
    assert _outside_is_zero(d, got_u, got_p)
    assert rel_err(d.to_vec(got_u, got_p), x) < 1e-10
    S.close()


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("beta", [0.0, 1e4])
def test_solve_reaches_the_direct_solution(ds, gamma, beta):
    """j = 3 (N = 32): solve to 1e-11 relative residual; the oracle's sparse direct solution of the
    L's bordered system, and the oracle's cycle count to the same tolerance (within one)."""
    j = 3
    d = ds[j]
    H = mg.Hierarchy(j + 1, beta, ds[:j + 1])
    _, _, f, g, _, F = _masked_state(d, 40)
    xo, hist = H.solve(F, mg.Params(gamma=gamma), tol=1e-11, max_cycles=100)
    xd = H.direct(F)
    S = _solver(j, beta, gamma=gamma)
    u, p, rep = S.solve(dev(f), dev(g), tol=1e-11, max_cycles=100)
    assert rep.converged and abs(rep.cycles - (len(hist) - 1)) <= 1, (rep.cycles, len(hist) - 1)
    assert rel_err(d.to_vec(host(u), host(p)), xd) < 1e-8
    assert abs(d.w @ host(p).ravel()[d.pnodes]) < 1e-12 * np.abs(host(p)).max()
    S.close()


@pytest.mark.parametrize("gamma", [1, 2])
def test_mixed_first_step_is_one_cycle(ds, gamma):
    """STOKES_MIXED on the L, j = 3: one refinement step from zero is one float32 cycle of the L
    (Sec. 3) added to the float64 iterate, then the zero-mean projection over the L: the oracle's
    float64 cycle to float32 accuracy, zero outside the L."""
    j, beta = 3, 1e4
    d = ds[j]
    H = mg.Hierarchy(j + 1, beta, ds[:j + 1])
    _, _, f, g, _, F = _masked_state(d, 50 + gamma)
    x = H.project_mean(j, H.cycle(j, np.zeros(d.ndof), F, mg.Params(gamma=gamma)))
    S = _solver(j, beta, gamma=gamma, precision="mixed")
    u, p, rep = S.solve(dev(f), dev(g), tol=1e-30, max_cycles=1)
    got_u, got_p = host(u), host(p)
    assert rep.cycles == 1 and not rep.converged
    assert _outside_is_zero(d, got_u, got_p)
    assert rel_err(d.to_vec(got_u, got_p), x) < 1e-5
    S.close()


@pytest.mark.parametrize("j", [3, 4])
@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("beta", [0.0, 1e4])
def test_mixed_solve_reaches_the_direct_solution(ds, j, gamma, beta):
    """STOKES_MIXED on the L: float32 cycles inside float64 iterative refinement reach the oracle's
    sparse direct solution to float64 accuracy (1e-11 relative residual), in the oracle's float64
    cycle count within two, with zero entries outside the L and a zero pressure mean over the L."""
    d = ds[j]
    H = mg.Hierarchy(j + 1, beta, ds[:j + 1])
    _, _, f, g, _, F = _masked_state(d, 60 + j)
    xo, hist = H.solve(F, mg.Params(gamma=gamma), tol=1e-11, max_cycles=100)
    xd = H.direct(F)
    S = _solver(j, beta, gamma=gamma, precision="mixed")
    u, p, rep = S.solve(dev(f), dev(g), tol=1e-11, max_cycles=100)
    got_u, got_p = host(u), host(p)
    assert rep.converged and abs(rep.cycles - (len(hist) - 1)) <= 2, (rep.cycles, len(hist) - 1)
    assert _outside_is_zero(d, got_u, got_p)
    assert rel_err(d.to_vec(got_u, got_p), xd) < 1e-8
    assert abs(d.w @ got_p.ravel()[d.pnodes]) < 1e-12 * np.abs(got_p).max()
    S.close()
