"""The cycle's kernels launched with programmatic dependent launch (STOKES_MG_PDL=1, read once per
process, so the solve runs in a child process) give the same solves as the default launches:
single mixed-precision and float64 solves and a small batch, against the oracle's exact discrete
solution and against each other."""
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
from paper_1502_04070_gb300.solver import Solver, BatchSolver
out = {}
for prec in ("mixed", "fp64"):
    k, beta = 5, 10.0
    fn, gn = workloads.random_nodal(k, 41)
    S = Solver(k + 1, beta, precision=prec)
    f, g = S.load_vectors(torch.from_numpy(fn).cuda(), torch.from_numpy(gn).cuda(), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-9, max_cycles=200)
    out[prec] = {"u": u.cpu().numpy().ravel().tolist(), "p": p.cpu().numpy().ravel().tolist(),
                 "cycles": rep.cycles, "rel": rep.rel_residual}
ks, betas = [3, 4, 5], [1.0, 1e3, 1e6]
fs, gs = [], []
for k, b in zip(ks, betas):
    fn, gn = workloads.random_nodal(k, 50 + k)
    S = Solver(k + 1, b, precision="mixed")
    f, g = S.load_vectors(torch.from_numpy(fn).cuda(), torch.from_numpy(gn).cuda(), project_g=True)
    fs.append(f); gs.append(g)
B = BatchSolver([k + 1 for k in ks], betas, precision="mixed", autotune=False)
us, ps, cyc, rel, st = B.solve(fs, gs, tol=1e-9, max_cycles=200)
out["batch"] = {"cycles": list(cyc), "rel": list(rel), "status": st}
print(json.dumps(out))
"""


def _run(pdl):
    env = dict(os.environ)
    env["STOKES_MG_PDL"] = pdl
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_programmatic_dependent_launch_gives_the_same_solves():
    on, off = _run("1"), _run("0")
    k, beta = 5, 10.0
    d = fem.discretizations(k + 1)[k]
    fn, gn = workloads.random_nodal(k, 41)
    F = d.load(fn, gn, project_g=True)
    xo = mg.direct_solve(d.system(beta), d, F)
    scale = np.abs(xo).max()
    for prec in ("mixed", "fp64"):
        a, b = on[prec], off[prec]
        assert a["cycles"] == b["cycles"], (prec, a["cycles"], b["cycles"])
        assert a["rel"] <= 1e-9 and b["rel"] <= 1e-9
        xa = np.concatenate([a["u"], a["p"]])
        xb = np.concatenate([b["u"], b["p"]])
        # launch order does not change any arithmetic: identical results
        assert np.array_equal(xa, xb), prec
        x = d.to_vec(np.asarray(a["u"]), np.asarray(a["p"]))
        assert np.abs(x - xo).max() <= 1e-6 * scale, prec
    assert on["batch"]["status"] == 0 and off["batch"]["status"] == 0
    assert on["batch"]["cycles"] == off["batch"]["cycles"]
    assert max(on["batch"]["rel"]) <= 1e-9
