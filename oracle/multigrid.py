"""Coupled multigrid for the generalized Stokes system, restated from the paper (Secs. 3-5).

Iteration (Sec. 3, eq. sm:comp and the coarse-grid correction that follows it):
    nu_pre smoothing steps, then  r_{k-1} = I_k^{k-1} (F_k - A_k x_k),  z_{k-1} ~ A_{k-1}^{-1} r_{k-1}
    by gamma recursive cycles from a zero start (gamma = 1: V-cycle, gamma = 2: W-cycle),
    x_k += I_{k-1}^k z_{k-1},  then nu_post smoothing steps.  On level 0 the coarse problem is
    solved exactly (Sec. 3).
Smoothers (Sec. 4):
    Uzawa type:  u^{m-1/2} = u^{m-1} + tau Ahat^{-1} (f - A u^{m-1} - B^T p^{m-1})
                 p^{m}     = p^{m-1} - sigma Shat^{-1} (g - B u^{m-1/2})
                 u^{m}     = u^{m-1} + tau Ahat^{-1} (f - A u^{m-1} - B^T p^{m})
    normal equation:  x^{m} = x^{m-1} + tau L^{-1} A L^{-1} (F - A x^{m-1})
with the practical preconditioner of Sec. 6 (eq. numintroduc):
    Ahat = diag A_k,   Shat = diag(B_k Ahat^{-1} B_k^T),   L = diag(Ahat, Shat),
    tau = sigma = 0.8 for Uzawa, tau = 0.35 for the normal equation (Sec. 6).
Readings where the paper is silent:
  * post-smoothing uses the same smoother as pre-smoothing;
  * the pressure space is the full P1 nodal space; zero mean is imposed by the projection
    p <- p - (w^T p)/(w^T 1), w = M_P 1, after every cycle, and the singular level-0 system is
    solved with that constraint as a border row/column (Sec. 1 requires int p = 0);
  * the initial guess is zero on the finest level and on every coarse correction;
  * the stopping test is the relative Euclidean residual ||F - A x|| / ||F|| on the unknowns.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, transfer

UZAWA = "uzawa"
NORMAL_EQ = "normal"


@dataclass
class Level:
    disc: fem.Discretization
    beta: float
    S: sp.csr_matrix = None          # [[A, B^T], [B, 0]]
    A: sp.csr_matrix = None
    B: sp.csr_matrix = None
    Ahat: np.ndarray = None          # diag A
    Shat: np.ndarray = None          # diag(B Ahat^{-1} B^T)
    P: sp.csr_matrix = None          # prolongation from the next coarser level (None on level 0)

    def __post_init__(self):
        d = self.disc
        self.A = d.A(self.beta)
        self.B = d.Bi
        self.S = d.system(self.beta)
        self.Ahat = self.A.diagonal().copy()
        self.Shat = np.asarray(self.B.multiply(self.B) @ (1.0 / self.Ahat)).ravel()

    @property
    def nu(self):
        return self.disc.nu

    def split(self, x):
        return x[:self.nu], x[self.nu:]


@dataclass
class Params:
    nu_pre: int = 3
    nu_post: int = 3
    tau: float = 0.8
    sigma: float = 0.8
    smoother: str = UZAWA
    gamma: int = 1


class Hierarchy:
    """All levels k = 0 .. levels-1 with their matrices, diagonals and transfers.  The multigrid
    iteration descends to `coarse_level` (default 0, the coarse mesh of Sec. 6), where the coarse
    problem is solved exactly (Sec. 3); the levels below it are not used."""

    def __init__(self, levels: int, beta: float, discs=None, coarse_level: int = 0):
        self.discs = discs if discs is not None else fem.discretizations(levels)
        self.levels = [Level(d, beta) for d in self.discs]
        for l in range(1, len(self.levels)):
            self.levels[l].P = transfer.prolongation(self.discs[l - 1], self.discs[l])
        self.beta = beta
        if not 0 <= coarse_level < len(self.levels):
            raise ValueError("coarse_level must lie in 0 .. levels - 1")
        self.coarse_level = coarse_level
        dc = self.discs[coarse_level]
        Sc = self.levels[coarse_level].S.toarray()
        n = Sc.shape[0]
        w = np.concatenate([np.zeros(dc.nu), dc.w])
        border = np.zeros((n + 1, n + 1))
        border[:n, :n] = Sc
        border[:n, n] = w
        border[n, :n] = w
        self.coarse_bordered = border

    @property
    def finest(self):
        return self.levels[-1]

    # ------------------------------------------------------------------ smoothers
    def uzawa_step(self, lvl: Level, x, F, prm: Params):
        """One step of the Uzawa-type smoother (Sec. 4), written as its three lines."""
        u, p = lvl.split(x)
        f, g = lvl.split(F)
        A, B = lvl.A, lvl.B
        u_half = u + prm.tau * (f - A @ u - B.T @ p) / lvl.Ahat
        p_new = p - prm.sigma * (g - B @ u_half) / lvl.Shat
        u_new = u + prm.tau * (f - A @ u - B.T @ p_new) / lvl.Ahat
        return np.concatenate([u_new, p_new])

    def normal_eq_step(self, lvl: Level, x, F, prm: Params):
        """One step of the preconditioned normal-equation smoother (Sec. 4) with L = diag(Ahat, Shat)."""
        Linv = 1.0 / np.concatenate([lvl.Ahat, lvl.Shat])
        r = F - lvl.S @ x
        return x + prm.tau * Linv * (lvl.S @ (Linv * r))

    def smooth(self, lvl, x, F, prm: Params):
        if prm.smoother == UZAWA:
            return self.uzawa_step(lvl, x, F, prm)
        if prm.smoother == NORMAL_EQ:
            return self.normal_eq_step(lvl, x, F, prm)
        raise ValueError(prm.smoother)

    # ------------------------------------------------------------------ coarse solve
    def coarse_solve(self, F0):
        """Exact solve on the coarsest level of the iteration (Sec. 3): the bordered system fixes
        w^T p = 0."""
        rhs = np.concatenate([F0, [0.0]])
        return np.linalg.solve(self.coarse_bordered, rhs)[:-1]

    # ------------------------------------------------------------------ cycle
    def cycle(self, l: int, x, F, prm: Params):
        """One multigrid iteration on level l (Sec. 3)."""
        if l == self.coarse_level:
            return self.coarse_solve(F)
        lvl = self.levels[l]
        for _ in range(prm.nu_pre):
            x = self.smooth(lvl, x, F, prm)
        r = F - lvl.S @ x
        rc = lvl.P.T @ r                                   # restriction = transposed embedding
        z = np.zeros(self.levels[l - 1].disc.ndof)
        for _ in range(prm.gamma):
            z = self.cycle(l - 1, z, rc, prm)
        x = x + lvl.P @ z
        for _ in range(prm.nu_post):
            x = self.smooth(lvl, x, F, prm)
        return x

    def project_mean(self, l: int, x):
        """p <- p - (w^T p)/(w^T 1), w = M_P 1: the representative of p in L^2_0 (Sec. 1)."""
        d = self.discs[l]
        x = x.copy()
        p = x[d.nu:]
        x[d.nu:] = p - (d.w @ p) / d.w.sum()
        return x

    def residual(self, l, x, F):
        return F - self.levels[l].S @ x

    def solve(self, F, prm: Params, tol=1e-10, max_cycles=100, x0=None):
        """Cycles from x0 (default 0) on the finest level until ||F - A x|| <= tol ||F||.
        Returns (x, history of residual norms including the initial one)."""
        L = len(self.levels) - 1
        x = np.zeros(len(F)) if x0 is None else x0.copy()
        nF = np.linalg.norm(F)
        hist = [np.linalg.norm(self.residual(L, x, F))]
        for _ in range(max_cycles):
            if hist[-1] <= tol * nF:
                break
            x = self.cycle(L, x, F, prm)
            x = self.project_mean(L, x)
            hist.append(np.linalg.norm(self.residual(L, x, F)))
        return x, np.array(hist)

    def direct(self, F, l=None):
        """Exact discrete solution with the zero-mean condition as a border (sparse direct)."""
        l = len(self.levels) - 1 if l is None else l
        return direct_solve(self.levels[l].S, self.discs[l], F)


def direct_solve(S, disc: fem.Discretization, F):
    n = S.shape[0]
    w = np.concatenate([np.zeros(disc.nu), disc.w])
    Sb = sp.bmat([[S, sp.csr_matrix(w[:, None])], [sp.csr_matrix(w[None, :]), None]]).tocsc()
    return spla.spsolve(Sb, np.concatenate([F, [0.0]]))[:n]


def smoother_conditions(lvl: Level, tau=0.8, sigma=0.8):
    """Diagnostic of the hypotheses of the smoothing analysis (Sec. 4, eq. def:tau:sigma):
    tau^-1 Ahat >= A  and  sigma^-1 Shat >= tau B Ahat^-1 B^T, i.e.
    lambda_max(Ahat^-1 A) <= 1/tau  and  lambda_max(Shat^-1 B Ahat^-1 B^T) <= 1/(sigma tau),
    by dense symmetric eigenvalues of the diagonally scaled matrices (small levels only).
    Returns the two largest eigenvalues and whether each condition holds."""
    A = lvl.A.toarray()
    d = 1.0 / np.sqrt(lvl.Ahat)
    lam_a = np.linalg.eigvalsh(d[:, None] * A * d[None, :])[-1]
    B = lvl.B.toarray()
    St = B @ (B.T / lvl.Ahat[:, None])
    e = 1.0 / np.sqrt(lvl.Shat)
    St = 0.5 * (St + St.T)
    lam_s = np.linalg.eigvalsh(e[:, None] * St * e[None, :])[-1]
    return {"lambda_A": lam_a, "lambda_S": lam_s,
            "A_condition": lam_a <= 1.0 / tau, "S_condition": lam_s <= 1.0 / (sigma * tau)}


def contraction(hist):
    """Per-cycle factors q_i = ||r_i|| / ||r_{i-1}|| and their geometric mean (Sec. 6 mean rate)."""
    hist = np.asarray(hist)
    q = hist[1:] / hist[:-1]
    n = len(q)
    qmean = (hist[-1] / hist[0]) ** (1.0 / n) if n else float("nan")
    return q, qmean
