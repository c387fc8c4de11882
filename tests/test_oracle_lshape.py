"""Pins of the oracle on the L-shaped domain (oracle/lshape.py): the unit square without
[1/2, 1]^2, where the method applies although the convergence theory (convex domains) does not
(Sec. 1).

* the meshes: 6 * 4^(j+1) triangles on level j, total area 3/4, every triangle inside the closed
  L and inside its parent;
* well-posedness: B^T has only the constant pressure in its kernel (dense SVD), although two
  corner triangles have all their vertices on the boundary;
* the Galerkin identity I^T A_j I = A_{j-1} of the masked transfers;
* V- and W-cycles converge to the sparse direct solution;
* Taylor-Hood orders 3, 2, 2 for a smooth manufactured solution vanishing on the whole boundary of
  the L (stream function with double zeros on the re-entrant sides);
* the square's canonical embedding restricted to the L's unknowns is the L's embedding.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, lshape
from oracle import multigrid as mg


@pytest.fixture(scope="module")
def ds():
    return lshape.discretizations(5)


def test_meshes(ds):
    for j, d in enumerate(ds):
        m = d.mesh
        assert len(m.tris) == 6 * 4 ** (j + 1)
        pts = m.verts[m.tris].astype(np.float64) / (2 * m.n)
        area, _ = fem.geometry(pts)
        assert np.all(area > 0) and abs(area.sum() - 0.75) < 1e-14
        inside = ~((pts[..., 0] > 0.5) & (pts[..., 1] > 0.5))
        assert np.all(inside)
        if j > 0:
            pm = ds[j - 1].mesh
            par = pm.verts[pm.tris[m.parent]].astype(np.float64) / (2 * pm.n)
            for c in range(3):
                q = pts[:, c]
                a, b, cc = par[:, 0], par[:, 1], par[:, 2]
                v0, v1, v2 = b - a, cc - a, q - a
                det = v0[:, 0] * v1[:, 1] - v0[:, 1] * v1[:, 0]
                l1 = (v2[:, 0] * v1[:, 1] - v2[:, 1] * v1[:, 0]) / det
                l2 = (v0[:, 0] * v2[:, 1] - v0[:, 1] * v2[:, 0]) / det
                assert np.all(np.stack([1 - l1 - l2, l1, l2]) >= -1e-14)


def test_pressure_kernel_is_the_constants(ds):
    for d in ds[:3]:
        Bt = d.Bi.T.toarray()
        s = sla.svdvals(Bt)
        assert np.sum(s < 1e-10 * s.max()) == 1
        assert np.abs(Bt @ np.ones(Bt.shape[1])).max() < 1e-13


def test_galerkin_identity(ds):
    for j in (1, 2, 3):
        H = mg.Hierarchy(j + 1, 10.0, ds[:j + 1])
        P = H.levels[j].P
        G = P.T @ H.levels[j].S @ P - H.levels[j - 1].S
        assert abs(G).max() < 1e-12


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("beta", [0.0, 1e4, 1e8])
def test_multigrid_converges_to_direct_solution(ds, beta, gamma):
    """Tolerance 1e-8 for beta = 1e8, where the float64 Euclidean residual levels off near 1e-9 on
    the square as well; 1e-10 otherwise."""
    j = 3
    d = ds[j]
    H = mg.Hierarchy(j + 1, beta, ds[:j + 1])
    rng = np.random.default_rng(4)
    F = rng.uniform(-1, 1, d.ndof)
    F[d.nu:] -= F[d.nu:].mean()
    tol = 1e-8 if beta >= 1e8 else 1e-10
    x, hist = H.solve(F, mg.Params(gamma=gamma), tol=tol, max_cycles=100)
    assert hist[-1] <= tol * np.linalg.norm(F)
    xd = H.direct(F)
    assert np.abs(x - xd).max() <= 1e3 * tol * np.abs(xd).max()


def _manufactured(beta):
    sy = pytest.importorskip("sympy")
    x, y = sy.symbols("x y")
    psi = (x * (1 - x) * y * (1 - y) * (x - sy.Rational(1, 2)) * (y - sy.Rational(1, 2))) ** 2
    ux, uy = sy.diff(psi, y), -sy.diff(psi, x)
    p = sy.cos(sy.pi * x) * sy.cos(sy.pi * y)
    lap = lambda w: sy.diff(w, x, 2) + sy.diff(w, y, 2)
    fx = -lap(ux) + beta * ux + sy.diff(p, x)
    fy = -lap(uy) + beta * uy + sy.diff(p, y)
    f = sy.lambdify((x, y), [fx, fy], "numpy")
    u = sy.lambdify((x, y), [ux, uy], "numpy")
    gu = sy.lambdify((x, y), [[sy.diff(ux, x), sy.diff(ux, y)], [sy.diff(uy, x), sy.diff(uy, y)]], "numpy")
    return f, u, gu


def test_manufactured_convergence_orders(ds):
    """||u - u_h||_L2 ~ h^3, |u - u_h|_H1 ~ h^2, ||p - p_h||_L2 ~ h^2 on the L.  The discrete p
    approximates -p (the sign of the weak form, Sec. 2) shifted to zero mean over the L:
    int_L cos(pi x) cos(pi y) = 0 - (int_{1/2}^1 cos(pi t) dt)^2 = -1/pi^2, mean -4/(3 pi^2)."""
    beta = 10.0
    f, u, gu = _manufactured(beta)
    shift = 4.0 / (3.0 * np.pi ** 2)
    exact_p = lambda X, Y: -(np.cos(np.pi * X) * np.cos(np.pi * Y) + shift)

    def bc(v, X):
        return v * np.ones_like(X) if np.isscalar(v) else v

    errs = []
    for j in (1, 2, 3):
        d = ds[j]
        n = d.n
        t = np.arange(2 * n + 1) / (2.0 * n)
        X, Y = np.meshgrid(t, t)
        fn = np.stack([bc(c, X) for c in f(X, Y)])
        F = d.load(fn, np.zeros((n + 1, n + 1)))
        x = mg.direct_solve(d.system(beta), d, F)
        uh, ph = d.from_vec(x)
        e = fem.error_norms(d, uh, ph,
                            lambda A, B_: [bc(c, A) for c in u(A, B_)],
                            lambda A, B_: [[bc(c, A) for c in row] for row in gu(A, B_)],
                            exact_p)
        errs.append(e)
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[-1] > np.array([2.7, 1.8, 1.7])), rates


def test_square_transfers_restrict_to_the_l(ds):
    """The L's canonical embedding (coarse L basis functions evaluated at the fine L nodes) equals
    the square's embedding restricted to the L's unknowns: the transfer kernels of the square can
    serve the L with a mask (a fine node of the L interpolates from coarse nodes of the L only)."""
    from oracle import transfer
    sq = fem.discretizations(5)
    for j in (0, 1, 2):
        Lc, Lf = ds[j], ds[j + 1]
        Sc, Sf = sq[j + 1], sq[j + 2]
        P_l = transfer.prolongation(Lc, Lf).toarray()
        P2, P1 = transfer.prolongation_full(Sc, Sf)
        P2, P1 = P2.toarray(), P1.toarray()
        ref_u = P2[Lf.interior][:, Lc.interior]
        ref_p = P1[Lf.pnodes][:, Lc.pnodes]
        niF, niC = Lf.ni, Lc.ni
        assert np.abs(P_l[:niF, :niC] - ref_u).max() < 1e-15
        assert np.abs(P_l[niF:2 * niF, niC:2 * niC] - ref_u).max() < 1e-15
        assert np.abs(P_l[2 * niF:, 2 * niC:] - ref_p).max() < 1e-15
        # a fine node of the L draws on no coarse node strictly inside the removed quadrant (only on
        # nodes of the closed L, whose re-entrant-side values are Dirichlet zeros), and a fine vertex
        # of the L only on coarse vertices of the L
        Xc, Yc = Sc.coords[:, 0], Sc.coords[:, 1]
        used = np.abs(P2[Lf.interior]).sum(axis=0) > 0
        assert not np.any(used & (Xc > Sc.n) & (Yc > Sc.n))
        used_p = np.flatnonzero(np.abs(P1[Lf.pnodes]).sum(axis=0) > 0)
        assert np.all(np.isin(used_p, Lc.pnodes))
