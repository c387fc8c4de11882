"""The experiment of Sec. 6 on the CUDA path: W(3,3) cycles with the Uzawa smoother from x^(0) = 0
on F = A x*, x* the L2 projection of the cone solution, with the error measured after every cycle
in the norm of eq. defMcL.  The oracle supplies x*, F and the norm; every cycle runs in the
library (one stokes_cycle call per iteration).

* k = 4, 5: the float64 error history equals the oracle's, cycle by cycle;
* k = 7, 8: the float64 history equals the one the oracle wrote
  (tests/golden/replication_w33_k78.json, from tests/golden/make_replication_golden.py), and the
  iteration counts lie within the band around the paper's Table 3
  (tests/golden/paper_tables_sec6.json) that the oracle's own counts meet on k = 4..6;
* k = 7, mixed precision (float32 W-cycles inside float64 refinement): the counts stay within
  one of the float64 ones and within the same band.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import experiments as ex
from oracle import fem
from oracle import multigrid as mg
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = json.load(open(os.path.join(HERE, "golden", "paper_tables_sec6.json")))
GOLD = json.load(open(os.path.join(HERE, "golden", "replication_w33_k78.json")))
BETAS = TABLES["betas"]
EPS = 1e-9


def band(n_paper):
    return max(2, math.ceil(n_paper / 4))


def paper_n(k, j):
    t = TABLES["table3"]
    return t["n"][t["k"].index(k)][j]


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(9)


@pytest.fixture(scope="module")
def projections(discs):
    return {}


def _xstar(discs, projections, k):
    if k not in projections:
        projections[k] = ex.l2_projection(discs[k])
    return projections[k]


def gpu_errors(d, k, beta, xs, precision="fp64", max_cycles=60):
    """The protocol of Sec. 6 with the library's cycle; returns (n, q, errors, divergent)."""
    from paper_1502_04070_gb300.solver import Solver
    F = d.system(beta) @ xs
    fu, gp = d.from_vec(F)
    S = Solver(k + 1, beta, gamma=2, precision=precision)
    try:
        f, g = dev(fu), dev(gp)
        u, p = S.zeros_u(), S.zeros_p()

        def step(_x):
            S.cycle(u, p, f, g)
            return d.to_vec(host(u), host(p))

        return ex.mean_rate(step, np.zeros_like(xs), xs, lambda e: ex.error_norm(d, beta, e),
                            max_cycles=max_cycles)
    finally:
        S.close()


def _near_threshold(errs):
    """True when the stopping decision of the reference history is within 10 % of the 1e-9 line
    (the tolerance of the history comparison below), where the count may move by one."""
    e0 = errs[0]
    n = len(errs) - 1
    return any(abs(errs[i] / (EPS * e0) - 1.0) < 0.1 for i in (n - 1, n) if i >= 1)


def _same_history(got, ref):
    n_g, _, eg, div_g = got
    n_r, eref = len(ref) - 1, np.asarray(ref)
    assert not div_g
    assert n_g == n_r or (abs(n_g - n_r) == 1 and _near_threshold(eref)), (n_g, n_r)
    m = min(n_g, n_r) + 1
    assert np.abs(eg[:m] - eref[:m]).max() <= 1e-10 * eref[0]


@pytest.mark.parametrize("k", [4, 5])
def test_fp64_matches_oracle_history(discs, projections, k):
    xs = _xstar(discs, projections, k)
    d = discs[k]
    for beta in BETAS:
        H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
        F = H.finest.S @ xs
        prm = mg.Params(gamma=2)
        step = lambda x: H.project_mean(k, H.cycle(k, x, F, prm))
        _, _, eo, div_o = ex.mean_rate(step, np.zeros_like(xs), xs, lambda e: ex.error_norm(d, beta, e))
        assert not div_o
        _same_history(gpu_errors(d, k, beta, xs), eo)


@pytest.mark.parametrize("k", [7, 8])
def test_fp64_table3_levels_7_8(discs, projections, k):
    xs = _xstar(discs, projections, k)
    d = discs[k]
    for j, run in enumerate(GOLD["levels"][str(k)]):
        assert run["beta"] == BETAS[j]
        got = gpu_errors(d, k, run["beta"], xs)
        _same_history(got, run["errors"])
        n_p = paper_n(k, j)
        assert abs(got[0] - n_p) <= band(n_p), (k, run["beta"], got[0], n_p)


def test_mixed_precision_table3_level_7(discs, projections):
    k = 7
    xs = _xstar(discs, projections, k)
    d = discs[k]
    for j, run in enumerate(GOLD["levels"][str(k)]):
        n, q, errs, div = gpu_errors(d, k, run["beta"], xs, precision="mixed")
        assert not div
        assert abs(n - run["n"]) <= 1, (run["beta"], n, run["n"])
        n_p = paper_n(k, j)
        assert abs(n - n_p) <= band(n_p), (run["beta"], n, n_p)
