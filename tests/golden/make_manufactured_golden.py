"""Writes tests/golden/manufactured_k8.json with the oracle's (and only the oracle's) cycle counts and
residual histories to 1e-8 relative residual (Uzawa smoother, Sec. 4, tau = sigma = 0.8, nu = 3+3,
zero start):

* the manufactured problem (u = curl(sin^2(pi x) sin^2(pi y)), p = cos(pi x) cos(pi y), beta = 1e4)
  on levels k = 4..8 with the V-cycle and the W-cycle (Sec. 3: gamma = 1, 2), each with the coarsest
  level 0 and 3 (exact solve there);
* the robustness sweep of h = 1/512 (k = 8, beta in {0, 1, 1e2, 1e4, 1e6, 1e8}, f and g uniform[-1,1]
  nodal, seed 1, g zero-mean) with the W-cycle, coarsest level 0 and 3 (the V-cycle counts are in
  sweep_k8.json).

Run:  python tests/golden/make_manufactured_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fem  # noqa: E402
from oracle import multigrid as mg  # noqa: E402
from paper_1502_04070_gb300 import workloads  # noqa: E402

BETAS = [0.0, 1.0, 1e2, 1e4, 1e6, 1e8]


def solve(ds, beta, F, gamma, tol=1e-8, coarse_level=0):
    k = len(ds) - 1
    t = time.time()
    H = mg.Hierarchy(k + 1, beta, ds, coarse_level=coarse_level)
    x, hist = H.solve(F, mg.Params(gamma=gamma), tol=tol, max_cycles=150)
    q, qm = mg.contraction(hist)
    out = {"k": k, "beta": beta, "gamma": gamma, "coarse_level": coarse_level, "cycles": len(hist) - 1,
           "mean_rate": float(qm), "rhs_norm": float(np.linalg.norm(F)), "history": hist.tolist(),
           "seconds": time.time() - t}
    print(k, beta, gamma, coarse_level, len(hist) - 1, qm, time.time() - t, flush=True)
    return out


if __name__ == "__main__":
    man = []
    ds_all = fem.discretizations(9)
    for k in range(4, 9):
        ds = ds_all[:k + 1]
        fn, gn = workloads.manufactured_nodal(k, 1e4)
        F = ds[-1].load(fn, gn, project_g=True)
        for gamma in (1, 2):
            man.append(solve(ds, 1e4, F, gamma))
            man.append(solve(ds, 1e4, F, gamma, coarse_level=3))
    fn, gn = workloads.random_nodal(8, 1)
    F = ds_all[-1].load(fn, gn, project_g=True)
    sweep = [solve(ds_all, b, F, 2) for b in BETAS]
    sweep_c3 = [solve(ds_all, b, F, 2, coarse_level=3) for b in BETAS]
    res = {"source": "oracle/ (CPU float64), written by tests/golden/make_manufactured_golden.py",
           "manufactured": {"beta": 1e4, "tol": 1e-8, "runs": man},
           "k8_sweep_w": {"k": 8, "seed": 1, "tol": 1e-8, "gamma": 2, "runs": sweep},
           "k8_sweep_w_c3": {"k": 8, "seed": 1, "tol": 1e-8, "gamma": 2, "coarse_level": 3, "runs": sweep_c3}}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "manufactured_k8.json"), "w") as fh:
        json.dump(res, fh, indent=1)
