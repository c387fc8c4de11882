"""The robustness sweep at full size (h = 1/512, k = 8, 2,356,227 unknowns) against values the
oracle wrote (tests/golden/sweep_k8.json, from tests/golden/make_sweep_golden.py):
cycle counts to 1e-8 and residual histories of the float64 path, and the mixed path's final
float64 residual, checked again by the oracle's own sparse matrix."""
import json
import os

import numpy as np
import pytest

from paper_1502_04070_gb300 import workloads
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sweep_k8.json")))


@pytest.fixture(scope="module")
def inputs():
    return workloads.random_nodal(8, 1)


@pytest.fixture(scope="module")
def oracle_k8():
    from oracle import fem
    return fem.discretizations(9)[-1]


@pytest.mark.parametrize("run", GOLD["k8_sweep"]["runs"], ids=lambda r: "beta=%g" % r["beta"])
def test_fp64_sweep_matches_oracle_history(inputs, run):
    from paper_1502_04070_gb300.solver import Solver
    fn, gn = inputs
    S = Solver(9, run["beta"])
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=100)
    assert rep.converged
    assert rep.cycles == run["cycles"]
    h = np.array(rep.history)
    ref = np.array(run["history"])
    assert np.abs(h - ref).max() <= 1e-7 * ref.max()
    assert abs(rep.rhs_norm - run["rhs_norm"]) <= 1e-12 * run["rhs_norm"]


@pytest.mark.parametrize("beta", [0.0, 1e4, 1e8])
def test_mixed_sweep_residual_checked_by_oracle(inputs, oracle_k8, beta):
    from paper_1502_04070_gb300.solver import Solver
    fn, gn = inputs
    S = Solver(9, beta, precision="mixed")
    f, g = S.load_vectors(dev(fn), dev(gn), project_g=True)
    u, p, rep = S.solve(f, g, tol=1e-8, max_cycles=100)
    assert rep.converged
    d = oracle_k8
    F = d.load(fn, gn, project_g=True)
    r = F - d.system(beta) @ d.to_vec(host(u), host(p))
    assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(F)
    gold = {r_["beta"]: r_["cycles"] for r_ in GOLD["k8_sweep"]["runs"]}[beta]
    assert abs(rep.cycles - gold) <= 2
