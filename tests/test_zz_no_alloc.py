"""stokes_residual_norm2_noalloc: the residual norm for callers that cannot allocate device memory
(it keeps its scratch in a fixed array inside the library).  Checked through the C-ABI against
the oracle's ||F - S x|| (assembled sparse matrix, float64) at k = 5, against the handle-based
stokes_residual_norm on two calls in a row, and at the largest size the fixed array is built for
(levels = 11, N = 2048).  This file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

from paper_1502_04070_gb300 import workloads

pytestmark = pytest.mark.gpu


def _host_inputs(k, seed):
    u, p = workloads.random_state(k, seed)
    f, g = workloads.random_nodal(k, seed + 1)
    return u, p, f, g - g.mean()


def _dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _noalloc(lib, k, beta, u, p, f, g):
    import torch
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = lib.stokes_residual_norm2_noalloc(k + 1, beta, ptr(u), ptr(p), ptr(f), ptr(g), ptr(out), None)
    torch.cuda.synchronize()
    return st, math.sqrt(float(out.item()))


def test_noalloc_residual_norm_matches_oracle():
    from oracle import fem
    from oracle import multigrid as mg
    from paper_1502_04070_gb300 import _binding
    lib = _binding.load()
    k, beta = 5, 1e3
    hu, hp, hf, hg = _host_inputs(k, 205)
    d = fem.discretizations(k + 1)[-1]
    lvl = mg.Level(d, beta)
    r = d.to_vec(hf, hg) - lvl.S @ d.to_vec(hu, hp)
    ref = float(np.linalg.norm(r))
    for _ in range(2):                                   # two calls in a row share the scratch array
        st, got = _noalloc(lib, k, beta, *_dev((hu, hp, hf, hg)))
        assert st == _binding.OK
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def test_noalloc_residual_norm_matches_handle_entry_point():
    from paper_1502_04070_gb300 import _binding
    from paper_1502_04070_gb300.solver import Solver
    lib = _binding.load()
    for k, beta in ((6, 1e3), (6, 1e3), (9, 0.0), (10, 1e4)):   # two calls in a row; k = 10 fills the array
        u, p, f, g = _dev(_host_inputs(k, 100 + k))
        S = Solver(k + 1, beta)
        ref = S.residual_norm(u, p, f, g)
        st, got = _noalloc(lib, k, beta, u, p, f, g)
        assert st == _binding.OK
        assert abs(got - ref) <= 1e-12 * ref, (k, got, ref)
        S.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_1502_04070_gb300 import _binding
    lib = _binding.load()
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    assert lib.stokes_residual_norm2_noalloc(12, 1.0, p, p, p, p, p, None) == _binding.ERR_BAD_ARG
    assert lib.stokes_residual_norm2_noalloc(0, 1.0, p, p, p, p, p, None) == _binding.ERR_BAD_ARG
