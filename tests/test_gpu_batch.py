"""Batched solves in one CUDA-graph launch (conditional WHILE nodes): every instance matches its
own single solve and the oracle's exact discrete solution."""
import numpy as np
import pytest

from oracle import fem
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_matches_oracle_and_single_solves(precision):
    import torch
    from paper_1502_04070_gb300.solver import BatchSolver, Solver
    ks, betas, seeds = workloads.batch_spec(10, 3, k_min=1, k_max=5)
    ds = fem.discretizations(max(ks) + 1)
    B = BatchSolver([k + 1 for k in ks], betas, precision=precision)
    fs, gs, nodal = [], [], []
    for k, beta, seed in zip(ks, betas, seeds):
        fn, gn = workloads.random_nodal(k, seed)
        S = Solver(k + 1, beta, precision=precision)
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        fs.append(f)
        gs.append(g)
        nodal.append((fn, gn, S))
    us, ps, cyc, rel, st = B.solve(fs, gs, tol=1e-9, max_cycles=300)
    assert st == 0
    assert max(rel) <= 1e-9
    for i, (k, beta) in enumerate(zip(ks, betas)):
        fn, gn, S = nodal[i]
        d = ds[k]
        F = d.load(fn, gn, project_g=True)
        x = d.to_vec(host(us[i]), host(ps[i]))
        r = F - d.system(beta) @ x
        assert np.linalg.norm(r) <= 1.0001e-9 * np.linalg.norm(F)
        xo = mg.direct_solve(d.system(beta), d, F)
        assert rel_err(x, xo) < 1e-5
        u1, p1, rep = S.solve(fs[i], gs[i], tol=1e-9, max_cycles=300)
        assert abs(rep.cycles - cyc[i]) <= 1
    # a second solve reuses the graph and gives the same answer
    us2, ps2, cyc2, rel2, st2 = B.solve(fs, gs, tol=1e-9, max_cycles=300, us=[torch.zeros_like(u) for u in us],
                                        ps=[torch.zeros_like(p) for p in ps])
    assert cyc2 == cyc
    for a, b_ in zip(us2, us):
        assert float((a - b_).abs().max()) <= 1e-12 * float(b_.abs().max())
    assert B.kernel_launches() > 0
