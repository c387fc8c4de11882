"""Writes tests/golden/sweep_k8.json with the oracle's (and only the oracle's) results for the
robustness sweep: h = 1/512 (k = 8), beta in {0, 1, 1e2, 1e4, 1e6, 1e8}, f and g with uniform[-1,1]
nodal values (seed 1, g shifted to zero mean), V(3,3) Uzawa cycles (Sec. 4, tau = sigma = 0.8) from
zero to 1e-8 relative residual.  Also h = 1/32 (k = 4), beta = 1, g = 0, seed 0, to 1e-10.

Run:  python tests/golden/make_sweep_golden.py
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


def run(k, betas, seed, with_g, tol):
    ds = fem.discretizations(k + 1)
    d = ds[-1]
    fn, gn = workloads.random_nodal(k, seed, with_g=with_g)
    F = d.load(fn, gn, project_g=True)
    out = []
    for beta in betas:
        t = time.time()
        H = mg.Hierarchy(k + 1, beta, ds)
        x, hist = H.solve(F, mg.Params(), tol=tol, max_cycles=100)
        q, qm = mg.contraction(hist)
        out.append({"beta": beta, "cycles": len(hist) - 1, "history": hist.tolist(),
                    "rhs_norm": float(np.linalg.norm(F)), "mean_rate": float(qm),
                    "seconds": time.time() - t})
        print(k, beta, len(hist) - 1, qm, time.time() - t, flush=True)
    return out


if __name__ == "__main__":
    res = {
        "source": "oracle/ (CPU float64), written by tests/golden/make_sweep_golden.py",
        "k8_sweep": {"k": 8, "seed": 1, "tol": 1e-8, "runs": run(8, BETAS, 1, True, 1e-8)},
        "k4_plain": {"k": 4, "seed": 0, "tol": 1e-10, "runs": run(4, [1.0], 0, False, 1e-10)},
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_k8.json"), "w") as fh:
        json.dump(res, fh, indent=1)
