"""A registered device allocator (stokes_set_allocator, the boundary's allocator callback): with
PyTorch's caching allocator registered, a solver's level buffers come from it (torch counts them as
allocated, and they return to it when the solver is destroyed), and the solve still meets the oracle's
exact discrete solution."""
import numpy as np
import pytest

from oracle import fem
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,coarse_level", [("mixed", 0), ("fp64", 2)])
def test_torch_caching_allocator_serves_the_solver(precision, coarse_level):
    import torch
    from paper_1502_04070_gb300.solver import Solver, use_torch_allocator
    k, beta = 4, 1e2
    d = fem.discretizations(k + 1)[-1]
    fn, gn = workloads.random_nodal(k, 41)
    F = d.load(fn, gn, project_g=True)
    xd = mg.Hierarchy(k + 1, beta, fem.discretizations(k + 1)).direct(F)
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    use_torch_allocator(True)
    try:
        S = Solver(k + 1, beta, precision=precision, coarse_level=coarse_level)
        torch.cuda.synchronize()
        m1 = torch.cuda.memory_allocated()
        # level slabs of k = 4 alone: 3 velocity and 4 vertex arrays of the finest level, float64
        n = 2 ** (k + 1)
        assert m1 - m0 >= 8 * (3 * 2 * (2 * n + 1) ** 2 + 4 * (n + 1) ** 2)
        f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
        u, p, rep = S.solve(f, g, tol=1e-11, max_cycles=100)
        assert rep.converged
        assert rel_err(d.to_vec(host(u), host(p)), xd) < 1e-8
        torch.cuda.synchronize()
        m_before_close = torch.cuda.memory_allocated()
        S.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == m_before_close - (m1 - m0)
    finally:
        use_torch_allocator(False)
