"""Planar float32 levels (stokes_params.tma_level): the float32 layout whose rows start on 16-byte
boundaries, and the one-kernel Uzawa step (Sec. 4) whose input tiles arrive by tensor-memory-access
box copies, against the oracle:

* nu float32 steps on a planar finest level equal the oracle's three-line steps within 2e-5 of the
  largest entry (float32 rounding of row sums of a few dozen terms) at k = 5, 6 (N + 1 = 2^(k+1) + 1
  cells per side fill no tile: ragged tiles at both ends, both mid-line bands, tiles whose boxes
  reach outside the arrays on every side) and several beta (k = 9: tests/test_gpu_oracle_k9.py);
* mixed-precision V and W cycles with planar levels from 5 up (so a planar level restricts to a
  compact one) converge to the oracle's direct solution with the oracle's cycle count (within one),
  with coarsest level 0 and 3;
* a planar hierarchy and an all-compact one solve the same problem in the same number of steps.
"""
import numpy as np
import pytest

from oracle import fem
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu

KMAX = 6


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(KMAX + 1)


def _state(k, seed):
    u, p = workloads.random_state(k, seed)
    f, g = workloads.random_nodal(k, seed + 1000)
    return u, p, f, g - g.mean()


@pytest.mark.parametrize("k", [5, 6])
@pytest.mark.parametrize("beta", [0.0, 1e2, 1e8])
@pytest.mark.parametrize("nu,variant", [(1, 0), (3, 0), (3, 1), (3, 2), (3, 3), (1, 4), (3, 4), (3, 5)])
def test_planar_step_by_oracle(discs, k, beta, nu, variant):
    """Every planar step variant: tiles for 3 or 4 resident CTAs per SM, with and without the L2
    prefetch of a later tile, and two cell rows per warp pass."""
    from paper_1502_04070_gb300.solver import Solver, planar_step_variant, set_planar_step_variant
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
    d = H.discs[-1]
    u, p, f, g = _state(k, 300 + k)
    # the oracle from the same float32-rounded inputs, in float64
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    x = d.to_vec(r32(u), r32(p))
    F = d.to_vec(r32(f), r32(g))
    for _ in range(nu):
        x = H.uzawa_step(H.finest, x, F, mg.Params())
    S = Solver(k + 1, beta, precision="mixed", tma_level=5)
    t = lambda a: dev(a).float().contiguous()
    tu, tp = t(u), t(p)
    old = planar_step_variant(k + 1)
    set_planar_step_variant(k + 1, variant)
    try:
        S.smooth_f32(tu, tp, t(f), t(g), nu)
    finally:
        set_planar_step_variant(k + 1, old)
    uo, po = d.from_vec(x)
    got = np.concatenate([host(tu.double()).ravel(), host(tp.double()).ravel()])
    ref = np.concatenate([uo.ravel(), po.ravel()])
    assert rel_err(got, ref) < 2e-5, rel_err(got, ref)
    S.close()


def test_planar_step_zeroes_the_boundary(discs):
    """Boundary velocity nodes come back zero whatever the caller's arrays hold there (the planar
    copy of the state is zero on the Dirichlet ring)."""
    from paper_1502_04070_gb300.solver import Solver
    k = 5
    u, p, f, g = _state(k, 77)
    u = u.copy()
    u[:, 0, :] = 1.0
    u[:, :, -1] = -2.0
    S = Solver(k + 1, 1e2, precision="mixed", tma_level=5)
    tu = dev(u).float().contiguous()
    tp = dev(p).float().contiguous()
    S.smooth_f32(tu, tp, dev(f).float().contiguous(), dev(g).float().contiguous(), 1)
    out = host(tu)
    assert np.all(out[:, 0, :] == 0) and np.all(out[:, -1, :] == 0)
    assert np.all(out[:, :, 0] == 0) and np.all(out[:, :, -1] == 0)
    S.close()


_DIRECT = {}


@pytest.mark.parametrize("gamma,coarse_level,variant", [(1, 0, 0), (2, 0, 1), (2, 3, 2), (1, 3, 3), (1, 0, 4), (2, 3, 5)])
def test_planar_mixed_solve_by_oracle(discs, gamma, coarse_level, variant):
    """k = 5 with levels 5 and up planar: the finest level restricts to a compact level."""
    from paper_1502_04070_gb300.solver import Solver, planar_step_variant, set_planar_step_variant
    k, beta = 5, 1e2
    d = discs[k]
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1], coarse_level=coarse_level)
    fn, gn = workloads.random_nodal(k, 90 + k)
    F = d.load(fn, gn, project_g=True)
    _, hist = H.solve(F, mg.Params(gamma=gamma), tol=1e-8, max_cycles=100)
    if k not in _DIRECT:
        _DIRECT[k] = H.direct(F)   # the finest system's solution: the same for every coarsest level
    xd = _DIRECT[k]
    old = planar_step_variant(k + 1)
    set_planar_step_variant(k + 1, variant)
    try:
        S = Solver(k + 1, beta, precision="mixed", gamma=gamma, coarse_level=coarse_level, tma_level=5)
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=100)
    finally:
        set_planar_step_variant(k + 1, old)
    assert rep.converged, rep
    assert abs(rep.cycles - (len(hist) - 1)) <= 1, (rep.cycles, len(hist) - 1)
    assert rel_err(d.to_vec(host(u), host(p)), xd) < 1e-6
    S.close()


@pytest.mark.parametrize("k,gamma,coarse_level,nu,variant", [(6, 1, 0, (3, 3), 0), (6, 2, 3, (3, 3), 5),
                                                          (6, 2, 0, (2, 1), 1), (5, 1, 3, (3, 3), 4),
                                                          (6, 1, 3, (3, 0), 2)])
def test_planar_first_refinement_step_is_one_cycle(discs, k, gamma, coarse_level, nu, variant):
    """One refinement step from zero with planar levels from 5 up is one float32 cycle (Sec. 3) and
    the zero-mean projection: the oracle's float64 cycle within 1e-5 of the largest entry.  With
    nu_post > 0 the coarse-grid correction of every planar level is added to the staged tiles of its
    first post-smoothing step (coarse level planar at k = 6, compact below); nu_post = 0 takes the
    separate prolongation kernel."""
    from paper_1502_04070_gb300.solver import Solver, planar_step_variant, set_planar_step_variant
    beta = 1e2
    d = discs[k]
    H = mg.Hierarchy(k + 1, beta, discs[:k + 1], coarse_level=coarse_level)
    fn, gn = workloads.random_nodal(k, 70 + k)
    F = d.load(fn, gn, project_g=True)
    prm = mg.Params(gamma=gamma, nu_pre=nu[0], nu_post=nu[1])
    x = H.project_mean(k, H.cycle(k, np.zeros(d.ndof), F, prm))
    olds = {lv: planar_step_variant(lv + 1) for lv in range(5, k + 1)}
    for lv in olds:
        set_planar_step_variant(lv + 1, variant)
    try:
        S = Solver(k + 1, beta, precision="mixed", gamma=gamma, coarse_level=coarse_level, tma_level=5,
                   nu_pre=nu[0], nu_post=nu[1])
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        u, p, rep = S.solve(f, g, tol=1e-30, max_cycles=1)
    finally:
        for lv, v in olds.items():
            set_planar_step_variant(lv + 1, v)
    assert rep.cycles == 1
    assert rel_err(d.to_vec(host(u), host(p)), x) < 1e-5
    S.close()


def test_planar_and_compact_hierarchies_agree(discs):
    """k = 7 (N = 256), manufactured-style random data: the solve with levels 5..7 planar and the
    solve with every level compact take the same steps, and both meet the tolerance in float64."""
    from paper_1502_04070_gb300.solver import Solver
    k, beta = 7, 1e4
    fn, gn = workloads.random_nodal(k, 5)
    out = {}
    for tl in (5, 14):
        S = Solver(k + 1, beta, precision="mixed", tma_level=tl)
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=100)
        assert rep.converged and rep.rel_residual <= 1e-8, rep
        out[tl] = (rep.cycles, np.concatenate([host(u).ravel(), host(p).ravel()]))
        S.close()
    assert abs(out[5][0] - out[14][0]) <= 1, (out[5][0], out[14][0])
    assert rel_err(out[5][1], out[14][1]) < 1e-6


@pytest.mark.parametrize("k", [5, 6])
@pytest.mark.parametrize("beta", [0.0, 1e4])
@pytest.mark.parametrize("tma_level", [5, 14])
def test_defect_restriction_by_oracle(discs, k, beta, tma_level):
    """I^T (F - S x) in float32 from the finest level to the next, against the oracle's assembled S
    and prolongation P (float64, from the same float32-rounded inputs); on a planar finest level
    (tma_level = 5) defect and restriction run in one kernel on staged tiles, with the coarse level
    planar (k = 6) or compact (k = 5); tma_level = 14 is the compact two-kernel path.  Bound as for
    the smoother (2e-5 of the largest entry)."""
    from oracle import transfer
    from paper_1502_04070_gb300.solver import Solver
    c, d = discs[k - 1], discs[k]
    P = transfer.prolongation(c, d)
    u, p, f, g = _state(k, 500 + k)
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    x = d.to_vec(r32(u), r32(p))
    F = d.to_vec(r32(f), r32(g))
    ref = P.T @ (F - d.system(beta) @ x)
    fo, go = c.from_vec(ref)
    S = Solver(k + 1, beta, precision="mixed", tma_level=tma_level)
    t = lambda a: dev(a).float().contiguous()
    fc, gc = S.residual_restrict_f32(t(u), t(p), t(f), t(g))
    got = np.concatenate([host(fc.double()).ravel(), host(gc.double()).ravel()])
    assert rel_err(got, np.concatenate([fo.ravel(), go.ravel()])) < 2e-5
    S.close()


@pytest.mark.parametrize("k,tma_level", [(5, 14), (5, 5), (7, 0)])
def test_two_inner_cycles_per_refinement_step(discs, k, tma_level):
    """Two float32 cycles per float64 refinement step (stokes_params.inner_cycles = 2, the headline's
    setting) against one (whose solves the tests above check against the oracle's direct solution):
    the same solution to 1e-6, in about half the refinement steps (each step contracts by about the
    square of one cycle's rate)."""
    from paper_1502_04070_gb300.solver import Solver
    beta = 1e4
    fn, gn = workloads.random_nodal(k, 110 + k)
    out = {}
    for inner in (1, 2):
        S = Solver(k + 1, beta, precision="mixed", coarse_level=3, inner_cycles=inner, tma_level=tma_level)
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=100)
        assert rep.converged and rep.rel_residual <= 1e-8, rep
        out[inner] = (rep.cycles, np.concatenate([host(u).ravel(), host(p).ravel()]))
        S.close()
    assert abs(out[2][0] - (out[1][0] + 1) // 2) <= 1, (out[2][0], out[1][0])
    assert rel_err(out[2][1], out[1][1]) < 1e-6
