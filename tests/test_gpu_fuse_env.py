"""The coarse-grid correction of planar float32 levels added inside their first post-smoothing
step (the default) against the separate prolongation kernel (STOKES_MG_FUSE_PROLONG=0, read once
per process, so each solve runs in a child process): mixed-precision V and W solves with planar
levels from 5 up reach the oracle's exact discrete solution either way, in the same number of
refinement steps within one (the two paths round differently in float32 only)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import fem
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1502_04070_gb300 import workloads
from paper_1502_04070_gb300.solver import Solver
out = {}
for k, gamma, cl in ((5, 1, 0), (5, 2, 3), (6, 1, 3), (6, 2, 0)):
    fn, gn = workloads.random_nodal(k, 43)
    S = Solver(k + 1, 1e2, precision="mixed", gamma=gamma, coarse_level=cl, tma_level=5)
    f, g = S.load_vectors(torch.from_numpy(fn).cuda(), torch.from_numpy(gn).cuda(), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-9, max_cycles=200)
    out["%d-%d-%d" % (k, gamma, cl)] = {"u": u.cpu().numpy().ravel().tolist(), "p": p.cpu().numpy().ravel().tolist(),
                                        "cycles": rep.cycles, "rel": rep.rel_residual}
    S.close()
print(json.dumps(out))
"""


def _run(fuse):
    env = dict(os.environ)
    env["STOKES_MG_FUSE_PROLONG"] = fuse
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_fused_and_separate_prolongation_give_the_same_solves():
    on, off = _run("1"), _run("0")
    assert on.keys() == off.keys()
    d = fem.discretizations(6)[5]
    fn, gn = workloads.random_nodal(5, 43)
    xo = mg.direct_solve(d.system(1e2), d, d.load(fn, gn, project_g=True))
    scale = np.abs(xo).max()
    for key in on:
        a, b = on[key], off[key]
        assert a["rel"] <= 1e-9 and b["rel"] <= 1e-9, (key, a["rel"], b["rel"])
        assert abs(a["cycles"] - b["cycles"]) <= 1, (key, a["cycles"], b["cycles"])
        xa = np.concatenate([a["u"], a["p"]])
        xb = np.concatenate([b["u"], b["p"]])
        assert np.abs(xa - xb).max() <= 1e-6 * np.abs(xb).max(), key
        if key.startswith("5-"):   # the oracle's exact discrete solution at k = 5
            x = d.to_vec(np.asarray(a["u"]), np.asarray(a["p"]))
            assert np.abs(x - xo).max() <= 1e-6 * scale, key
