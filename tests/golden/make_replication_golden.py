"""Writes tests/golden/replication_w33_k78.json with the oracle's (and only the oracle's) results
for the experiment of Sec. 6 on levels k = 7 and 8: W(3,3) cycles with the Uzawa smoother
(tau = sigma = 0.8) from x^(0) = 0 on the L2 projection x* of the cone solution, the error
|||x^(i) - x*|||_k of eq. defMcL after every cycle until its reduction by 1e-9, and the mean rate
q, for beta in {0, 1e2, 1e4, 1e6, 1e8, 1e10} (the columns of Tables 2 and 3).

Run:  python tests/golden/make_replication_golden.py      (a few minutes on one core)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import experiments as ex  # noqa: E402
from oracle import fem  # noqa: E402
from oracle import multigrid as mg  # noqa: E402

BETAS = [0.0, 1e2, 1e4, 1e6, 1e8, 1e10]


def main():
    out = {"protocol": "Sec. 6: W(3,3), Uzawa tau = sigma = 0.8, x0 = 0, error norm of eq. defMcL with "
                       "h = sqrt(2)/N, stop at 1e-9 error reduction", "betas": BETAS, "levels": {}}
    for k in (7, 8):
        discs = fem.discretizations(k + 1)
        d = discs[k]
        xs = ex.l2_projection(d)
        runs = []
        for beta in BETAS:
            t = time.time()
            H = mg.Hierarchy(k + 1, beta, discs)
            F = H.finest.S @ xs
            prm = mg.Params(gamma=2)
            step = lambda x: H.project_mean(k, H.cycle(k, x, F, prm))
            n, q, errs, div = ex.mean_rate(step, np.zeros_like(xs), xs, lambda e: ex.error_norm(d, beta, e))
            runs.append({"beta": beta, "n": n, "q": q, "divergent": bool(div), "errors": errs.tolist()})
            print("k=%d beta=%g n=%d q=%.4f (%.1fs)" % (k, beta, n, q, time.time() - t), flush=True)
        out["levels"][str(k)] = runs
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "replication_w33_k78.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
