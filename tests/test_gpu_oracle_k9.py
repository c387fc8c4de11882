"""The CUDA path at h = 1/1024 (k = 9, 9,431,043 unknowns) checked by the oracle's own assembled
matrices, at the largest level the oracle assembles in about a minute (its CSR system holds about
2.4e8 nonzeros here).

* the load vectors of the device equal the oracle's (float64, 1e-12);
* the mixed-precision solve (float32 cycles with the step variants the autotuner picks at these
  sizes, float64 refinement) meets ||F - S x|| <= 1e-8 ||F|| with the oracle's S, and its pressure
  has zero mean (Sec. 1);
* one float32 Uzawa step (Sec. 4) equals the oracle's three-line step element by element within
  2e-5 of the largest entry (float32 rounding of sums of a few dozen terms): the step of the planar
  levels (tiles staged by tensor-memory-access copies; the default at this size) and every compact
  step variant that the autotuner chooses among at the large levels.
"""
import numpy as np
import pytest

from oracle import fem
from oracle import mesh as meshmod
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu

K = 9
BETA = 1e4


@pytest.fixture(scope="module")
def level():
    d = fem.Discretization(meshmod.hierarchy(K + 1)[-1])
    return d, mg.Level(d, BETA)


def test_k9_mixed_solve_residual_by_oracle(level):
    from paper_1502_04070_gb300.solver import Solver
    d, L = level
    fn, gn = workloads.random_nodal(K, 9)
    F = d.load(fn, gn, project_g=True)
    S = Solver(K + 1, BETA, precision="mixed")
    S.autotune()
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    assert rel_err(d.to_vec(host(f), host(g)), F) < 1e-12
    u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=200)
    assert rep.converged, rep
    x = d.to_vec(host(u), host(p))
    r = F - L.S @ x
    assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(F), np.linalg.norm(r) / np.linalg.norm(F)
    xp = x[d.nu:]
    assert abs(d.w @ xp) <= 1e-12 * (d.w @ np.abs(xp))
    S.close()


def _variants():
    # the three-kernel step, the pair tiles and the register-coefficient tiles (the autotuner's
    # candidates that win at k >= 8)
    return [4, 7, 8, 10, 11]


@pytest.mark.parametrize("variant", ["planar", None] + _variants())
def test_k9_float32_step_by_oracle(level, variant):
    from paper_1502_04070_gb300.solver import Solver, set_step_variant, step_variant
    d, L = level
    u, p = workloads.random_state(K, 31)
    f, g = workloads.random_nodal(K, 32)
    g = g - g.mean()
    # "planar": the finest level in the planar layout (the default here); otherwise every level compact
    S = Solver(K + 1, BETA, precision="mixed", tma_level=0 if variant == "planar" else 14)
    if variant in (None, "planar"):
        S.autotune()                     # the variant chosen for this size in this process
        variant = step_variant(K + 1)
    t = lambda a: dev(a).float().contiguous()
    tu, tp, tf, tg = t(u), t(p), t(f), t(g)
    old = step_variant(K + 1)
    set_step_variant(K + 1, variant)
    try:
        S.smooth_f32(tu, tp, tf, tg, 1)
    finally:
        set_step_variant(K + 1, old)
    # the oracle step from the same float32-rounded inputs, in float64
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    x = mg.Hierarchy.uzawa_step(None, L, d.to_vec(r32(u), r32(p)), d.to_vec(r32(f), r32(g)), mg.Params())
    uo, po = d.from_vec(x)
    got = np.concatenate([host(tu.double()).ravel(), host(tp.double()).ravel()])
    ref = np.concatenate([uo.ravel(), po.ravel()])
    assert rel_err(got, ref) < 2e-5, (variant, rel_err(got, ref))
    S.close()
