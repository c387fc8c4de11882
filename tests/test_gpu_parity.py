"""CUDA path vs the CPU oracle, element by element, through the C-ABI (float64 path).

Sizes k = 0..6 span many 32x8 thread tiles with ragged edges (N + 1 = 2^(k+1) + 1 cells per side)
and both mesh orientations with their mid-line seams.  Tolerance: float64 rounding of sums of at
most a few dozen terms, 1e-12 relative to the largest entry for single applications and 1e-10 for
whole cycles (the bound the plain float64 path must meet).
"""
import numpy as np
import pytest

from oracle import fem
from oracle import multigrid as mg
from oracle import transfer
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu

KMAX = 6


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(KMAX + 1)


@pytest.fixture(scope="module")
def Solver():
    from paper_1502_04070_gb300.solver import Solver
    return Solver


def _state(k, seed):
    u, p = workloads.random_state(k, seed)
    f, g = workloads.random_nodal(k, seed + 1000)
    g = g - g.mean()
    return u, p, f, g


@pytest.mark.parametrize("k", range(KMAX + 1))
@pytest.mark.parametrize("beta", [0.0, 1.0, 1e4, 1e8])
def test_residual(discs, Solver, k, beta):
    d = discs[k]
    u, p, f, g = _state(k, 10 + k)
    S = Solver(k + 1, beta)
    ru, rp = S.residual(dev(u), dev(p), dev(f), dev(g))
    r = d.to_vec(f, g) - d.system(beta) @ d.to_vec(u, p)
    ru_o, rp_o = d.from_vec(r)
    got = np.concatenate([host(ru).ravel(), host(rp).ravel()])
    ref = np.concatenate([ru_o.ravel(), rp_o.ravel()])
    assert rel_err(got, ref) < 1e-12
    nrm = S.residual_norm(dev(u), dev(p), dev(f), dev(g))
    assert abs(nrm - np.linalg.norm(r)) < 1e-12 * np.linalg.norm(r)


@pytest.mark.parametrize("k", [0, 2, 5])
@pytest.mark.parametrize("project", [False, True])
def test_load_vectors(discs, Solver, k, project):
    d = discs[k]
    rng = np.random.default_rng(20 + k)
    fn = rng.uniform(-1, 1, (2, 2 * d.n + 1, 2 * d.n + 1))     # boundary values included
    gn = rng.uniform(-1, 1, (d.n + 1, d.n + 1))
    S = Solver(k + 1, 1.0)
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=project)
    F = d.load(fn, gn, project_g=project)
    fo, go = d.from_vec(F)
    assert rel_err(host(f), fo) < 1e-13
    assert rel_err(host(g), go) < 1e-13
    if project:
        assert abs(host(g).sum()) < 1e-14 * np.abs(go).sum()


@pytest.mark.parametrize("k", [1, 3, 6])
@pytest.mark.parametrize("beta", [0.0, 1e3, 1e8])
@pytest.mark.parametrize("smoother", ["uzawa", "normal"])
def test_smoother(discs, Solver, k, beta, smoother):
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
    d = H.discs[-1]
    u, p, f, g = _state(k, 30 + k)
    prm = mg.Params(smoother=smoother, tau=0.8 if smoother == "uzawa" else 0.35)
    x = d.to_vec(u, p)
    F = d.to_vec(f, g)
    for _ in range(3):
        x = H.smooth(H.finest, x, F, prm)
    S = Solver(k + 1, beta, smoother=smoother)
    tu, tp = dev(u), dev(p)
    S.smooth(tu, tp, dev(f), dev(g), 3)
    uo, po = d.from_vec(x)
    assert rel_err(np.concatenate([host(tu).ravel(), host(tp).ravel()]),
                   np.concatenate([uo.ravel(), po.ravel()])) < 1e-11


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_transfers(discs, Solver, k):
    c, fz = discs[k - 1], discs[k]
    P = transfer.prolongation(c, fz)
    rng = np.random.default_rng(40 + k)
    ru, rp = workloads.random_state(k, 41 + k)
    S = Solver(k + 1, 1.0)
    fc, gc = S.restrict(dev(ru), dev(rp))
    ref = P.T @ fz.to_vec(ru, rp)
    fo, go = c.from_vec(ref)
    assert rel_err(np.concatenate([host(fc).ravel(), host(gc).ravel()]),
                   np.concatenate([fo.ravel(), go.ravel()])) < 1e-13
    uc, pc = workloads.random_state(k - 1, 42 + k)
    u0, p0 = workloads.random_state(k, 43 + k)
    tu, tp = dev(u0), dev(p0)
    S.prolong_add(dev(uc), dev(pc), tu, tp)
    x = fz.to_vec(u0, p0) + P @ c.to_vec(uc, pc)
    uo, po = fz.from_vec(x)
    assert rel_err(np.concatenate([host(tu).ravel(), host(tp).ravel()]),
                   np.concatenate([uo.ravel(), po.ravel()])) < 1e-13


@pytest.mark.parametrize("k", [1, 2, 4, 6])
@pytest.mark.parametrize("beta", [1.0, 1e6])
@pytest.mark.parametrize("gamma,smoother", [(1, "uzawa"), (2, "uzawa"), (1, "normal")])
def test_cycle(discs, Solver, k, beta, gamma, smoother):
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
    d = H.discs[-1]
    u, p, f, g = _state(k, 50 + k)
    prm = mg.Params(gamma=gamma, smoother=smoother, tau=0.8 if smoother == "uzawa" else 0.35)
    x = d.to_vec(u, p)
    F = d.to_vec(f, g)
    S = Solver(k + 1, beta, gamma=gamma, smoother=smoother)
    tu, tp = dev(u), dev(p)
    tf, tg = dev(f), dev(g)
    for _ in range(2):
        x = H.project_mean(k, H.cycle(k, x, F, prm))
        S.cycle(tu, tp, tf, tg)
    uo, po = d.from_vec(x)
    assert rel_err(np.concatenate([host(tu).ravel(), host(tp).ravel()]),
                   np.concatenate([uo.ravel(), po.ravel()])) < 1e-10


def test_solve_plain_fp64_h32(discs, Solver):
    """Plain method, float64: h = 1/32 (k = 4), beta = 1, f uniform[-1,1] nodal (seed 0), g = 0,
    V(3,3) Uzawa cycles to 1e-10 relative residual; the iterate, the cycle count and the residual
    history match the oracle."""
    k, beta = workloads.level_of_h(32), 1.0
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
    d = H.discs[-1]
    fn, gn = workloads.random_nodal(k, 0, with_g=False)
    F = d.load(fn, gn, project_g=True)
    x, hist = H.solve(F, mg.Params(), tol=1e-10, max_cycles=60)
    S = Solver(k + 1, beta)
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-10, max_cycles=60)
    assert rep.converged and rep.cycles == len(hist) - 1
    assert rel_err(rep.history, hist) < 1e-8
    uo, po = d.from_vec(x)
    assert rel_err(np.concatenate([host(u).ravel(), host(p).ravel()]),
                   np.concatenate([uo.ravel(), po.ravel()])) < 1e-10
    # the oracle's own residual of the GPU solution
    r = F - d.system(beta) @ d.to_vec(host(u), host(p))
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(F) * 1.0001


@pytest.mark.parametrize("beta", [1.0, 1e4])
def test_solve_mixed_precision(discs, Solver, beta):
    """float32 cycles inside float64 refinement reach 1e-8 relative residual in float64; the error
    against the oracle's exact discrete solution is reported in the assertion message."""
    k = 5
    if k > KMAX:
        pytest.skip()
    d = discs[k]
    fn, gn = workloads.random_nodal(k, 3)
    S = Solver(k + 1, beta, precision="mixed")
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=60)
    assert rep.converged
    F = d.load(fn, gn, project_g=True)
    xo = mg.direct_solve(d.system(beta), d, F)
    x = d.to_vec(host(u), host(p))
    r = F - d.system(beta) @ x
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(F) * 1.0001
    err = rel_err(x, xo)
    assert err < 1e-5, err


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6])
@pytest.mark.parametrize("beta", [0.0, 1e3, 1e8])
@pytest.mark.parametrize("nu", [1, 3])
def test_smoother_float32_fused(discs, Solver, k, beta, nu):
    """The fused one-kernel float32 Uzawa step of the mixed-precision path against the float64
    oracle.  Bound: float32 rounding of row sums of about 30 terms, measured relative to the
    largest entry of the result (2e-5)."""
    import torch
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
    d = H.discs[-1]
    u, p, f, g = _state(k, 70 + k)
    x = d.to_vec(u, p)
    F = d.to_vec(f, g)
    for _ in range(nu):
        x = H.uzawa_step(H.finest, x, F, mg.Params())
    S = Solver(k + 1, beta, precision="mixed")
    t = lambda a: dev(a).float().contiguous()
    tu, tp = t(u), t(p)
    S.smooth_f32(tu, tp, t(f), t(g), nu)
    uo, po = d.from_vec(x)
    got = np.concatenate([host(tu.double()).ravel(), host(tp.double()).ravel()])
    ref = np.concatenate([uo.ravel(), po.ravel()])
    assert rel_err(got, ref) < 2e-5


@pytest.mark.parametrize("k", [3, 5, 6])
@pytest.mark.parametrize("variant", range(12))
def test_smoother_float32_every_variant(discs, Solver, k, variant):
    """Every float32 step variant the autotuner may choose (four fused tile shapes, the three-kernel
    step with three block shapes, the component-pair tiles in three shapes, the register-coefficient
    tiles in two) gives the oracle's three
    Uzawa steps at a size whose cells do not fill the last tile or block (N + 1 = 2^(k+1) + 1 per
    side); at k = 6 the pair tiles take both their interior and their general path.  Bound as
    above (2e-5)."""
    from paper_1502_04070_gb300.solver import set_step_variant, step_variant
    beta = 1e2
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
    d = H.discs[-1]
    u, p, f, g = _state(k, 170 + k)
    x = d.to_vec(u, p)
    F = d.to_vec(f, g)
    for _ in range(3):
        x = H.uzawa_step(H.finest, x, F, mg.Params())
    S = Solver(k + 1, beta, precision="mixed", tma_level=14)   # every level on the compact variants
    t = lambda a: dev(a).float().contiguous()
    tu, tp = t(u), t(p)
    old = step_variant(k + 1)
    set_step_variant(k + 1, variant)
    try:
        S.smooth_f32(tu, tp, t(f), t(g), 3)
    finally:
        set_step_variant(k + 1, old)
    uo, po = d.from_vec(x)
    got = np.concatenate([host(tu.double()).ravel(), host(tp.double()).ravel()])
    ref = np.concatenate([uo.ravel(), po.ravel()])
    assert rel_err(got, ref) < 2e-5


@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("nu_pre,nu_post,gamma", [(3, 3, 2), (4, 3, 2), (3, 2, 1)])
def test_mixed_cycle_variants(discs, Solver, k, nu_pre, nu_post, gamma):
    """W-cycles and odd smoothing counts (the float32 ping-pong ends in the scratch buffer) in the
    mixed path converge to the oracle's exact discrete solution.  (nu = 2+1 is not tested: like
    2+2 in Sec. 6, Table 1, it diverges.)"""
    d = discs[k]
    fn, gn = workloads.random_nodal(k, 80 + k)
    S = Solver(k + 1, 10.0, precision="mixed", nu_pre=nu_pre, nu_post=nu_post, gamma=gamma)
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-9, max_cycles=300)
    F = d.load(fn, gn, project_g=True)
    xo = mg.direct_solve(d.system(10.0), d, F)
    assert rep.converged, rep
    assert rel_err(d.to_vec(host(u), host(p)), xo) < 1e-6


def test_divergence_is_reported(Solver):
    """Sec. 6, Table 1: the Uzawa smoother with nu = 1+1 diverges; the solver must stop with
    STOKES_DIVERGED instead of running to max_cycles or raising."""
    from paper_1502_04070_gb300 import _binding
    k = 4
    fn, gn = workloads.random_nodal(k, 90)
    S = Solver(k + 1, 1.0, nu_pre=1, nu_post=1)
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-9, max_cycles=400)
    assert rep.status == _binding.DIVERGED
