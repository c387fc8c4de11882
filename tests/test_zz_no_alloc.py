"""stokes_residual_norm2_noalloc: the residual norm for callers that cannot allocate device memory
(it keeps its scratch in a fixed array inside the library).  Checked through the C-ABI against the
handle-based stokes_residual_norm on two calls in a row; this file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

from paper_1502_04070_gb300 import workloads

pytestmark = pytest.mark.gpu


def _inputs(k, seed):
    import torch
    u, p = workloads.random_state(k, seed)
    f, g = workloads.random_nodal(k, seed + 1)
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (u, p, f, g - g.mean())]


def test_noalloc_residual_norm_matches_handle_entry_point():
    import torch
    from paper_1502_04070_gb300 import _binding
    from paper_1502_04070_gb300.solver import Solver
    lib = _binding.load()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    for k, beta in ((6, 1e3), (6, 1e3), (9, 0.0)):      # two calls in a row on the same size first
        u, p, f, g = _inputs(k, 100 + k)
        S = Solver(k + 1, beta)
        ref = S.residual_norm(u, p, f, g)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st = lib.stokes_residual_norm2_noalloc(k + 1, beta, ptr(u), ptr(p), ptr(f), ptr(g), ptr(out), None)
        assert st == _binding.OK
        torch.cuda.synchronize()
        got = math.sqrt(float(out.item()))
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
