"""The iteration's coarsest level above the coarse mesh (Sec. 3: exact solve on the coarsest level;
stokes_params.coarse_level = c > 0, a dense float64 inverse of the bordered level-c system computed on
the device by Gauss-Jordan elimination) against the oracle's hierarchy with the same coarsest level:

* whole V and W cycles in float64 element by element (1e-10), including c = k - 1, where one cycle
  is the exact two-grid correction;
* mixed-precision W-cycles with c = 3 converge to the oracle's direct solution with the oracle's
  cycle count, also after stokes_set_beta rebuilt the inverse for another beta.
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
    return fem.discretizations(7)


def _state(k, seed):
    u, p = workloads.random_state(k, seed)
    f, g = workloads.random_nodal(k, seed + 1000)
    return u, p, f, g - g.mean()


@pytest.mark.parametrize("k,c", [(2, 1), (3, 2), (4, 2), (4, 3), (5, 3)])
@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("beta", [1.0, 1e6])
def test_cycle_with_coarse_level(discs, k, c, gamma, beta):
    from paper_1502_04070_gb300.solver import Solver
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1], coarse_level=c)
    d = H.discs[-1]
    u, p, f, g = _state(k, 60 + k)
    prm = mg.Params(gamma=gamma)
    x = d.to_vec(u, p)
    F = d.to_vec(f, g)
    S = Solver(k + 1, beta, gamma=gamma, coarse_level=c)
    tu, tp, tf, tg = dev(u), dev(p), dev(f), dev(g)
    for _ in range(2):
        x = H.project_mean(k, H.cycle(k, x, F, prm))
        S.cycle(tu, tp, tf, tg)
    uo, po = d.from_vec(x)
    assert rel_err(np.concatenate([host(tu).ravel(), host(tp).ravel()]),
                   np.concatenate([uo.ravel(), po.ravel()])) < 1e-10
    S.close()


def test_mixed_w_cycle_with_coarse_level_3(discs):
    from paper_1502_04070_gb300.solver import Solver
    k = 5
    fn, gn = workloads.random_nodal(k, 77)
    d = discs[k]
    F = d.load(fn, gn, project_g=True)
    S = Solver(k + 1, 1e2, precision="mixed", gamma=2, coarse_level=3)
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    for beta in (1e2, 1e6):
        if beta != S.beta:
            S.set_beta(beta)
        H = mg.Hierarchy(k + 1, beta, discs[:k + 1], coarse_level=3)
        xo, hist = H.solve(F, mg.Params(gamma=2), tol=1e-8, max_cycles=60)
        u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=60)
        assert rep.converged and abs(rep.cycles - (len(hist) - 1)) <= 1, (beta, rep.cycles, len(hist) - 1)
        xd = H.direct(F)
        assert rel_err(d.to_vec(host(u), host(p)), xd) < 1e-6
    S.close()
