"""Pins of the oracle's multigrid against the paper's compact smoother form, the exact discrete
solution, Taylor-Hood convergence orders, and the robustness the paper proves and reports."""
import numpy as np
import pytest

from oracle import adjoint, fem
from oracle import multigrid as mg
from paper_1502_04070_gb300 import workloads


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(5)


def _rhs(d, seed):
    rng = np.random.default_rng(seed)
    F = rng.uniform(-1, 1, d.ndof)
    F[d.nu:] -= F[d.nu:].mean()
    return F


@pytest.mark.parametrize("beta", [0.0, 1.0, 1e6])
def test_uzawa_step_equals_compact_form(discs, beta):
    """Sec. 4: the Uzawa step is x <- x + Ahat_c^{-1}(F - A x) with
    Ahat_c = [[Ahat/tau, B^T], [B, tau B Ahat^{-1} B^T - Shat/sigma]]."""
    H = mg.Hierarchy(3, beta, discs[:3])
    lvl = H.finest
    tau, sigma = 0.8, 0.8
    Ah = np.diag(lvl.Ahat)
    B = lvl.B.toarray()
    Sh = np.diag(lvl.Shat)
    Ac = np.block([[Ah / tau, B.T], [B, tau * B @ np.diag(1 / lvl.Ahat) @ B.T - Sh / sigma]])
    rng = np.random.default_rng(1)
    x = rng.standard_normal(lvl.disc.ndof)
    F = rng.standard_normal(lvl.disc.ndof)
    ref = x + np.linalg.solve(Ac, F - lvl.S @ x)
    got = H.uzawa_step(lvl, x, F, mg.Params(tau=tau, sigma=sigma))
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


def test_diagonals_definition(discs):
    """Sec. 6 (eq. numintroduc): Shat = diag(B diag(A)^{-1} B^T), checked with dense algebra."""
    H = mg.Hierarchy(3, 7.0, discs[:3])
    lvl = H.finest
    A = lvl.A.toarray()
    B = lvl.B.toarray()
    assert np.allclose(lvl.Ahat, np.diag(A), rtol=0, atol=1e-15)
    S = B @ np.diag(1.0 / np.diag(A)) @ B.T
    assert np.abs(lvl.Shat - np.diag(S)).max() < 1e-14 * np.abs(S).max()


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("beta", [0.0, 1.0, 1e4, 1e8])
def test_multigrid_converges_to_direct_solution(discs, gamma, beta):
    H = mg.Hierarchy(4, beta, discs[:4])
    d = H.discs[-1]
    F = _rhs(d, 2)
    xd = H.direct(F)
    # attainable relative residual in float64: rounding of S x scales with |S| |x|
    floor = 50 * np.finfo(float).eps * np.linalg.norm(abs(H.finest.S) @ abs(xd)) / np.linalg.norm(F)
    tol = max(1e-12, floor)
    x, hist = H.solve(F, mg.Params(gamma=gamma), tol=tol, max_cycles=80)
    assert hist[-1] <= tol * np.linalg.norm(F)
    assert np.abs(x - xd).max() <= 1e3 * tol * np.abs(xd).max()
    assert abs(d.w @ x[d.nu:]) < 1e-13 * np.abs(x).max()        # zero mean pressure (Sec. 1)


def test_two_grid_exact_coarse(discs):
    """k = 1: the coarse problem is solved exactly (Sec. 3, eq. method:cga); the iterate equals
    smoothing + I A_0^{-1} I^T (F - A x) with A_0^{-1} from the sparse direct solver."""
    H = mg.Hierarchy(2, 1.0, discs[:2])
    F = _rhs(H.discs[1], 3)
    prm = mg.Params(nu_pre=2, nu_post=0)
    x = np.zeros_like(F)
    for _ in range(2):
        x = H.uzawa_step(H.finest, x, F, prm)
    r = F - H.finest.S @ x
    rc = H.finest.P.T @ r
    z = mg.direct_solve(H.levels[0].S, H.discs[0], rc)
    ref = x + H.finest.P @ z
    got = H.cycle(1, np.zeros_like(F), F, prm)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("c", [1, 2])
def test_coarse_level_is_an_exact_two_grid_solve(discs, c):
    """With the coarsest level of the iteration at c = k - 1 (Sec. 3: the coarse problem is solved
    exactly), one cycle is smoothing plus the exact coarse correction with A_c^{-1} taken from the
    sparse direct solver of the bordered level-c system."""
    k = c + 1
    H = mg.Hierarchy(k + 1, 3.0, discs[:k + 1], coarse_level=c)
    F = _rhs(H.discs[k], 5)
    prm = mg.Params(nu_pre=2, nu_post=0)
    x = np.zeros_like(F)
    for _ in range(2):
        x = H.uzawa_step(H.finest, x, F, prm)
    rc = H.finest.P.T @ (F - H.finest.S @ x)
    ref = x + H.finest.P @ mg.direct_solve(H.levels[c].S, H.discs[c], rc)
    got = H.cycle(k, np.zeros_like(F), F, prm)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("beta", [0.0, 1e4])
def test_w_cycle_with_finer_coarse_level_converges_to_direct_solution(discs, beta):
    """A W-cycle that stops at level 2 (an exact solve there) converges to the exact discrete
    solution, like the one that descends to level 0."""
    H = mg.Hierarchy(5, beta, discs, coarse_level=2)
    d = H.discs[-1]
    F = _rhs(d, 6)
    xd = H.direct(F)
    x, hist = H.solve(F, mg.Params(gamma=2), tol=1e-11, max_cycles=80)
    assert hist[-1] <= 1e-11 * np.linalg.norm(F)
    assert np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max()
    with pytest.raises(ValueError):
        mg.Hierarchy(3, beta, discs[:3], coarse_level=3)


def _contraction_estimate(H, k, gamma, its=25, seed=0):
    """Power iteration on the cycle's error propagation (F = 0, zero-mean pressure kept): the
    last ratio ||x_{m+1}|| / ||x_m|| estimates its spectral radius."""
    rng = np.random.default_rng(seed)
    x = H.project_mean(k, rng.uniform(-1, 1, H.discs[k].ndof))
    x /= np.linalg.norm(x)
    F = np.zeros_like(x)
    for _ in range(its):
        y = H.project_mean(k, H.cycle(k, x, F, mg.Params(gamma=gamma)))
        q = np.linalg.norm(y)
        x = y / q
    return q


def test_w_cycle_contraction_is_h_robust_and_the_v_cycle_is_not():
    """Sec. 3 proves h- and beta-independent convergence of the W-cycle (Sec. 6 runs W; it calls the
    V-cycle comparable).  On this mesh (beta = 0, Uzawa 3+3) the W-cycle's contraction levels off
    (0.380, 0.394, 0.394 at k = 5, 6, 7) while the V-cycle's grows (0.378, 0.394, then 0.55 at k = 7),
    which is why the V-cycle needs 68 cycles at h = 1/512 and 34 at h = 1/2048 in the benchmark."""
    ds = fem.discretizations(8)
    qw, qv = {}, {}
    for k in (5, 6, 7):
        H = mg.Hierarchy(k + 1, 0.0, ds[:k + 1])
        qw[k] = _contraction_estimate(H, k, 2)
        if k in (5, 7):
            qv[k] = _contraction_estimate(H, k, 1)
    assert all(0.3 < q < 0.42 for q in qw.values()), qw
    assert max(qw.values()) - min(qw.values()) < 0.03, qw
    assert qv[5] < 0.42 and qv[7] > 0.5, qv


def test_manufactured_convergence_orders():
    """Taylor-Hood P2-P1 (Sec. 2): ||u-u_h||_L2 ~ h^3, |u-u_h|_H1 ~ h^2, ||p-p_h||_L2 ~ h^2.
    The weak form of Sec. 2 carries +(p, div v), i.e. the discrete p approximates -p of the strong
    form -Lap u + beta u + grad p = f; the error is taken against -p."""
    for beta in (1.0, 1e4):
        errs = []
        ds = fem.discretizations(5)
        for k in (2, 3, 4):
            d = ds[k]
            fn, gn = workloads.manufactured_nodal(k, beta)
            F = d.load(fn, gn)
            S = d.system(beta)
            x = mg.direct_solve(S, d, F)
            u, p = d.from_vec(x)
            e = fem.error_norms(d, u, p, workloads.exact_u, workloads.exact_grad_u,
                                lambda X, Y: -workloads.exact_p(X, Y))
            errs.append(e)
        errs = np.array(errs)
        rates = np.log2(errs[:-1] / errs[1:])
        assert np.all(rates[-1] > np.array([2.7, 1.8, 1.7])), (beta, rates)


def test_robust_contraction(discs):
    """Sec. 4/5: contraction bounded independently of h and beta (V-cycle, Uzawa 3+3)."""
    counts = []
    for k in (2, 3, 4):
        for beta in (0.0, 1.0, 1e2, 1e4, 1e6, 1e8):
            H = mg.Hierarchy(k + 1, beta, discs[:k + 1])
            F = _rhs(H.discs[-1], 4)
            x, hist = H.solve(F, mg.Params(), tol=1e-8, max_cycles=60)
            q, qm = mg.contraction(hist)
            assert qm < 0.45, (k, beta, qm)
            counts.append(len(hist) - 1)
    assert max(counts) <= 2.5 * min(counts) + 2


def test_table1_structure(discs):
    """Sec. 6, Table 1 (k = 4): the Uzawa smoother diverges for nu = 1+1 and 2+2 and converges for
    3+3; the normal-equation smoother (tau = 0.35) already converges for 1+1."""
    H = mg.Hierarchy(5, 1.0, discs)
    F = _rhs(H.discs[-1], 5)
    for nu, ok in ((1, False), (2, False), (3, True)):
        x, hist = H.solve(F, mg.Params(gamma=2, nu_pre=nu, nu_post=nu), tol=1e-9, max_cycles=25)
        assert (hist[-1] < 1e-8 * hist[0]) == ok
    x, hist = H.solve(F, mg.Params(gamma=2, nu_pre=1, nu_post=1, smoother=mg.NORMAL_EQ, tau=0.35),
                      tol=1e-6, max_cycles=200)
    assert hist[-1] <= 1e-6 * hist[0]


def test_adjoint_vs_finite_differences(discs):
    """dL/dF and dL/dbeta of L = 1/2 ||u - u_t||_M^2 through the exact solve, against central
    differences (L is quadratic in F, so FD in F is exact up to rounding)."""
    beta = 30.0
    d = discs[3]
    H = mg.Hierarchy(4, beta, discs[:4])
    F = _rhs(d, 6)
    ut = np.random.default_rng(7).uniform(-1, 1, d.nu)
    lossgrad = lambda x: adjoint.loss_velocity_mass(d, x, ut)[1]
    x, gF, gb = adjoint.solve_and_gradients(H, F, lossgrad)

    def L(F_, beta_):
        Hb = mg.Hierarchy(4, beta_, discs[:4])
        return adjoint.loss_velocity_mass(d, Hb.direct(F_), ut)[0]

    rng = np.random.default_rng(8)
    for _ in range(3):
        dF = rng.standard_normal(d.ndof)
        dF[d.nu:] -= dF[d.nu:].mean()
        eps = 1e-3
        fd = (L(F + eps * dF, beta) - L(F - eps * dF, beta)) / (2 * eps)
        assert abs(fd - gF @ dF) < 1e-8 * max(1.0, abs(fd))
    eps = 1e-4 * beta
    fd = (L(F, beta + eps) - L(F, beta - eps)) / (2 * eps)
    assert abs(fd - gb) < 1e-6 * max(abs(fd), 1e-12)


@pytest.mark.parametrize("beta", [0.0, 1e4, 1e8])
def test_smoother_condition_diagnostic(discs, beta):
    """The diagnostic of the smoothing hypotheses (Sec. 4): each largest eigenvalue of a diagonally
    scaled SPD matrix lies between its mean diagonal, 1, and the Gershgorin bound max_i
    sum_j |M_ij| / M_ii; with tau = sigma = 0.8 neither condition holds on this mesh (lambda_A
    1.69-2.19 > 1.25, lambda_S 1.95 > 1.5625 at k = 3), as observed."""
    H = mg.Hierarchy(4, beta, discs[:4])
    lvl = H.finest
    c = mg.smoother_conditions(lvl)
    A = abs(lvl.A).toarray()
    g_a = (A.sum(axis=1) / lvl.Ahat).max()
    B = lvl.B.toarray()
    St = abs(B @ (B.T / lvl.Ahat[:, None]))
    g_s = (St.sum(axis=1) / lvl.Shat).max()
    assert 1.0 <= c["lambda_A"] <= g_a and 1.0 <= c["lambda_S"] <= g_s
    assert not c["A_condition"] and not c["S_condition"]
