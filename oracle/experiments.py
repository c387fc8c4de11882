"""The numerical experiment of Sec. 6: the cone-based exact solution, its L2 projection x* into
X_k, the error norm |||.|||_k of eq. defMcL and the mean convergence rate q.

TEST INFRASTRUCTURE (part of the oracle package): only tests, the smoke check and the benchmark's
CPU baseline may import it.

Sec. 6 chooses f and g so that the discrete solution on level k is the L2 projection of
    u(x, y) = phi(x, y) (y - 1/2, 1/2 - x),   p(x, y) = phi(x, y),
    phi(x, y) = max{0, min{1, 2 - 4 r}},  r = |(x, y) - (1/2, 1/2)|,
i.e. F_k = A_k x* with x* = (Pi_U u, Pi_P p).  The iteration starts from x^(0), stops at the first
n with |||x^(n) - x*|||_k <= eps |||x^(0) - x*|||_k (eps = 1e-9), and reports
q = (|||x^(n) - x*|||_k / |||x^(0) - x*|||_k)^(1/n).

Readings where the paper is silent:
  * x^(0) = 0;
  * |||.|||_k is the norm of eq. defMcL, L_k = diag((h^-2 + beta) M_U, h^-2 (beta + h^-2)^-1 M_P),
    with h = h_k the longest edge of the level-k mesh (Sec. 2: sqrt(2)/N on these meshes);
  * P_k is the zero-mean subspace of P1 (Sec. 1), so Pi_P p is the P1 projection minus its mean
    (constants lie in P1, and the zero-mean subspace is their orthogonal complement);
  * an iteration is "divergent" when the error grows beyond 1e6 times the initial error or does
    not reach the reduction within the cycle limit.
The load integrals use a collapsed Gauss rule per triangle; triangles that the kink circles of phi
(r = 1/4 and r = 1/2) cross are split into sub x sub sub-triangles first.  The mass systems are
solved by diagonally preconditioned conjugate gradients to a relative residual of 1e-14.
"""
import numpy as np

from . import fem

EPS = 1e-9


def cone(x, y):
    """phi of Sec. 6: 1 for r <= 1/4, 2 - 4r for 1/4 <= r <= 1/2, 0 beyond."""
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2)
    return np.maximum(0.0, np.minimum(1.0, 2.0 - 4.0 * r))


def cone_solution(x, y):
    """(u_x, u_y, p) of the Sec. 6 experiment at points (x, y)."""
    ph = cone(x, y)
    return ph * (y - 0.5), ph * (0.5 - x), ph


CONE_KINKS = (0.25, 0.5)


def composite_rule(sub, npts):
    """Collapsed Gauss rule on each of the sub^2 congruent sub-triangles of the reference triangle.
    Returns barycentric points (3, q) and weights summing to 1/2."""
    lam, w = fem._collapsed_gauss(npts)
    ref = lam[1:].T                                  # (q, 2) reference coordinates (xi1, xi2)
    pts, wts = [], []
    for i in range(sub):
        for j in range(sub - i):
            corners = [np.array([[i, j], [i + 1, j], [i, j + 1]])]
            if i + j + 1 < sub:
                corners.append(np.array([[i + 1, j], [i + 1, j + 1], [i, j + 1]]))
            for c in corners:
                c = c / sub
                xi = c[0] + ref[:, :1] * (c[1] - c[0]) + ref[:, 1:] * (c[2] - c[0])
                pts.append(xi)
                wts.append(w / sub ** 2)
    xi = np.concatenate(pts)
    return np.stack([1.0 - xi[:, 0] - xi[:, 1], xi[:, 0], xi[:, 1]]), np.concatenate(wts)


def _crossing(pts, radii, centre=(0.5, 0.5)):
    """Triangles (nt, 3, 2) whose distance range from the centre may contain one of the radii:
    the range over a triangle lies in [min over vertices - longest edge, max over vertices]."""
    r = np.sqrt((pts[..., 0] - centre[0]) ** 2 + (pts[..., 1] - centre[1]) ** 2)
    e = np.max(np.sqrt(((pts - np.roll(pts, 1, axis=1)) ** 2).sum(-1)), axis=1)
    lo, hi = r.min(1) - e, r.max(1)
    out = np.zeros(len(pts), bool)
    for c in radii:
        out |= (lo <= c) & (c <= hi)
    return out


def load_integrals(disc: fem.Discretization, fun, kinks=CONE_KINKS, npts=5, sub=8):
    """b_u = (u, phi_i) for every P2 node of the lattice (both components) and b_p = (p, psi_i) for
    every vertex, by quadrature; fun(x, y) -> (u_x, u_y, p).  Returns bx, by (n2,), bp (nv,)."""
    m = disc.mesh
    n = m.n
    pts = m.verts[m.tris].astype(np.float64) / (2 * n)
    area, _ = fem.geometry(pts)
    lat2 = fem.lattice_index_of(m)[m.tri_p2]                       # (nt, 6)
    latv = ((m.verts[:, 1] // 2) * (n + 1) + m.verts[:, 0] // 2)[m.tris]   # (nt, 3)
    bx, by, bp = np.zeros(disc.n2), np.zeros(disc.n2), np.zeros(disc.nv)
    kinked = _crossing(pts, kinks) if kinks else np.zeros(len(pts), bool)
    for sel, (lam, wq) in ((~kinked, fem._collapsed_gauss(npts)), (kinked, composite_rule(sub, 4))):
        idx = np.flatnonzero(sel)
        if len(idx) == 0:
            continue
        phi = np.stack([fem.evaluate_poly(p, lam) for p in fem.p2_basis()])   # (6, q)
        for c0 in range(0, len(idx), 8192):
            t = idx[c0:c0 + 8192]
            xq = np.einsum('iq,tic->tqc', lam, pts[t])
            ux, uy, pp = fun(xq[..., 0], xq[..., 1])
            W = 2.0 * area[t, None] * wq[None, :]
            bx += np.bincount(lat2[t].ravel(), ((W * ux) @ phi.T).ravel(), disc.n2)
            by += np.bincount(lat2[t].ravel(), ((W * uy) @ phi.T).ravel(), disc.n2)
            bp += np.bincount(latv[t].ravel(), ((W * pp) @ lam.T).ravel(), disc.nv)
    return bx, by, bp


def mass_solve(M, b, rtol=1e-14, max_iter=1000):
    """Solves M x = b for a symmetric positive definite mass matrix by conjugate gradients with the
    diagonal as preconditioner (mass matrices are spectrally equivalent to their diagonal, so the
    iteration count does not grow with the level).  Raises if the relative residual stays above
    rtol."""
    dinv = 1.0 / M.diagonal()
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    d = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for _ in range(max_iter):
        if np.linalg.norm(r) <= rtol * nb:
            return x
        Md = M @ d
        a = rz / (d @ Md)
        x += a * d
        r -= a * Md
        z = dinv * r
        rz, rz_old = r @ z, rz
        d = z + (rz / rz_old) * d
    if np.linalg.norm(b - M @ x) > 10 * rtol * nb:
        raise RuntimeError("mass_solve did not converge")
    return x


def l2_projection(disc: fem.Discretization, fun=cone_solution, kinks=CONE_KINKS):
    """x* = (Pi_U u, Pi_P p) as an unknown vector [u_x(interior); u_y(interior); p(vertices)]:
    M_U Pi_U u = (u, phi_i) on the interior P2 nodes, M_P q = (p, psi_i), Pi_P p = q - mean(q)."""
    bx, by, bp = load_integrals(disc, fun, kinks)
    I = disc.interior
    ux = mass_solve(disc.Mi, bx[I])
    uy = mass_solve(disc.Mi, by[I])
    q = mass_solve(disc.MP, bp)
    q = q - (disc.w @ q) / disc.w.sum()
    return np.concatenate([ux, uy, q])


def mesh_size(disc: fem.Discretization):
    """h_k = length of the longest edge (Sec. 2): the hypotenuse sqrt(2)/N of the right triangles."""
    return np.sqrt(2.0) / disc.n


def error_norm(disc: fem.Discretization, beta, e):
    """|||e|||_k = (L_k e, e)^(1/2) with L_k of eq. defMcL."""
    h2 = mesh_size(disc) ** -2
    eu, ep = e[:disc.nu], e[disc.nu:]
    Mi = disc.Mi
    ni = disc.ni
    uu = eu[:ni] @ (Mi @ eu[:ni]) + eu[ni:] @ (Mi @ eu[ni:])
    pp = ep @ (disc.MP @ ep)
    return np.sqrt((h2 + beta) * uu + h2 / (beta + h2) * pp)


def mean_rate(step, x0, xs, norm, eps=EPS, max_cycles=60, blowup=1e6):
    """Sec. 6 protocol: iterate x <- step(x) from x0 until norm(x - xs) <= eps norm(x0 - xs).
    Returns (n, q, errors, divergent); errors[i] = norm(x^(i) - xs)."""
    x = x0.copy()
    errs = [norm(x - xs)]
    for _ in range(max_cycles):
        x = step(x)
        errs.append(norm(x - xs))
        if errs[-1] <= eps * errs[0]:
            break
        if not np.isfinite(errs[-1]) or errs[-1] > blowup * errs[0]:
            break
    n = len(errs) - 1
    divergent = not (errs[-1] <= eps * errs[0])
    q = (errs[-1] / errs[0]) ** (1.0 / n) if np.isfinite(errs[-1]) else float("inf")
    return n, q, np.array(errs), divergent
