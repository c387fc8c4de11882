"""The cooperative small-level cycle (stokes_params.coop_level): the float32 V- or W-cycle from a small
level down to the coarsest level of the iteration (Sec. 3), its exact coarsest solve included, as one
cooperative launch whose phases meet at grid barriers, against the oracle:

* mixed-precision solves whose float32 cycle runs entirely in one launch (coop_level = the finest
  level, every level compact) converge to the oracle's direct solution (1e-6) with the oracle's
  cycle count (within one), for V and W cycles, coarsest levels 0, 2 and 3, and odd smoothing counts
  (the ping-pong of the last level ends in its scratch buffer);
* with the default planar levels (from level 6) and the cooperative cycle from level 5 down, and
  with the cooperative cycle off, k = 6 solves take the same number of steps and agree to 1e-6;
* one refinement step with the cooperative cycle equals one with a launch per phase to float32
  rounding (V and W, coarsest levels 0 and 3, odd smoothing counts).
"""
import numpy as np
import pytest

from oracle import fem
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(6)


_DIRECT = {}


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("gamma,coarse_level,nu_pre,nu_post", [(1, 0, 3, 3), (2, 0, 3, 3), (2, 3, 3, 3),
                                                                (1, 3, 3, 2), (2, 2, 4, 3)])
def test_coop_solve_by_oracle(discs, k, gamma, coarse_level, nu_pre, nu_post):
    from paper_1502_04070_gb300.solver import Solver
    beta = 1e2
    d = discs[k]
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1], coarse_level=coarse_level)
    fn, gn = workloads.random_nodal(k, 70 + k)
    F = d.load(fn, gn, project_g=True)
    # odd smoothing counts converge slowly with the V-cycle (rate about 0.88 at k = 5): room for it
    _, hist = H.solve(F, mg.Params(gamma=gamma, nu_pre=nu_pre, nu_post=nu_post), tol=1e-8, max_cycles=300)
    if k not in _DIRECT:
        _DIRECT[k] = H.direct(F)
    S = Solver(k + 1, beta, precision="mixed", gamma=gamma, coarse_level=coarse_level, nu_pre=nu_pre,
               nu_post=nu_post, tma_level=14, coop_level=k)
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=300)
    assert rep.converged, rep
    assert abs(rep.cycles - (len(hist) - 1)) <= 1, (rep.cycles, len(hist) - 1)
    assert rel_err(d.to_vec(host(u), host(p)), _DIRECT[k]) < 1e-6
    S.close()


@pytest.mark.parametrize("gamma,coarse_level", [(1, 0), (1, 3), (2, 3)])
def test_coop_matches_per_phase_launches(gamma, coarse_level):
    from paper_1502_04070_gb300.solver import Solver
    k, beta = 6, 1e4
    fn, gn = workloads.random_nodal(k, 12)
    out = {}
    for cl in (5, -1):
        S = Solver(k + 1, beta, precision="mixed", gamma=gamma, coarse_level=coarse_level, coop_level=cl)
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=100)
        assert rep.converged and rep.rel_residual <= 1e-8, rep
        out[cl] = (rep.cycles, np.concatenate([host(u).ravel(), host(p).ravel()]))
        S.close()
    assert abs(out[5][0] - out[-1][0]) <= 1, (out[5][0], out[-1][0])
    assert rel_err(out[5][1], out[-1][1]) < 1e-6


@pytest.mark.parametrize("k", [4, 6])
@pytest.mark.parametrize("gamma,coarse_level,nu_pre,nu_post", [(1, 3, 3, 2), (2, 0, 3, 3), (2, 3, 4, 3)])
def test_coop_cycle_equals_per_phase_launches(k, gamma, coarse_level, nu_pre, nu_post):
    """One mixed refinement step (stokes_cycle) with the float32 cycle as one cooperative launch and as
    one launch per phase, from the same state: the same arithmetic in a different order, equal to
    float32 rounding (1e-5 of the largest entry)."""
    from paper_1502_04070_gb300.solver import Solver
    fn, gn = workloads.random_nodal(k, 80 + k)
    out = []
    for cl in (k, -1):
        S = Solver(k + 1, 1e3, precision="mixed", gamma=gamma, coarse_level=coarse_level, nu_pre=nu_pre,
                   nu_post=nu_post, tma_level=14, coop_level=cl)
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        u, p = S.zeros_u(), S.zeros_p()
        S.cycle(u, p, f, g)
        out.append(np.concatenate([host(u).ravel(), host(p).ravel()]))
        S.close()
    assert rel_err(out[0], out[1]) < 1e-5
