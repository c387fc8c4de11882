"""Taylor-Hood P2-P1 finite element matrices by exact polynomial integration (Sec. 2).

The bilinear forms are those of the variational problem of Sec. 2 (eq. gen:bil):
    a(u, v) = (grad u, grad v) + beta (u, v)        -> A_k = K + beta M_U (one block per component)
    b(u, q) = (div u, q)                            -> B_k[i, j] = (div phi_j, psi_i)
and the block matrix of eq. gen:bil:mv is  [[A_k, B_k^T], [B_k, 0]].

Basis functions are written from their definitions in barycentric coordinates lambda_0..2:
    P2 vertex i:       lambda_i (2 lambda_i - 1)
    P2 edge (i, j):    4 lambda_i lambda_j
    P1 vertex i:       lambda_i
Integrals of monomials use the exact formula
    int_T lambda_0^a lambda_1^b lambda_2^c dx = 2|T| a! b! c! / (a + b + c + 2)!
so every element matrix is exact (no quadrature error).

Velocity unknowns are the P2 nodes off the boundary (u = 0 on the boundary, Sec. 1); pressure
unknowns are all P1 vertices, with the zero-mean condition imposed outside the matrix (see
multigrid.project_mean).  All global numbering is the canonical lattice order: P2 node (X, Y) has
flat index Y*(2N+1)+X, vertex (x, y) has flat index y*(N+1)+x.
"""
from functools import lru_cache
from math import factorial

import numpy as np
import scipy.sparse as sp

from . import mesh as meshmod

# ---------------------------------------------------------------- barycentric polynomials
# A polynomial is a dict {(a, b, c): coefficient} in lambda_0, lambda_1, lambda_2.


def _mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
            out[e] = out.get(e, 0.0) + ca * cb
    return out


def _d(p, i):
    """Partial derivative with respect to lambda_i."""
    out = {}
    for e, c in p.items():
        if e[i] > 0:
            f = list(e)
            f[i] -= 1
            f = tuple(f)
            out[f] = out.get(f, 0.0) + c * e[i]
    return out


def _unit(i):
    e = [0, 0, 0]
    e[i] = 1
    return tuple(e)


def monomial_integral_over_2area(e):
    """int_T lambda^e dx / (2|T|)."""
    a, b, c = e
    return factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)


def _int(p):
    return sum(c * monomial_integral_over_2area(e) for e, c in p.items())


def evaluate_poly(p, lam):
    """Value of polynomial p at barycentric point(s) lam = (lambda_0, lambda_1, lambda_2)
    (scalars or arrays of equal shape)."""
    return sum(c * lam[0] ** e[0] * lam[1] ** e[1] * lam[2] ** e[2] for e, c in p.items())


def p2_basis():
    """Local P2 basis in the node order v0, v1, v2, m12, m02, m01."""
    out = []
    for i in range(3):
        # lambda_i (2 lambda_i - 1)
        out.append(_mul({_unit(i): 1.0}, {_unit(i): 2.0, (0, 0, 0): -1.0}))
    for (i, j) in ((1, 2), (0, 2), (0, 1)):
        out.append(_mul({_unit(i): 4.0}, {_unit(j): 1.0}))
    return out


def p1_basis():
    return [{_unit(i): 1.0} for i in range(3)]


def evaluate_p2(lam):
    """Values of the 6 local P2 basis functions at barycentric point lam."""
    return np.array([evaluate_poly(p, lam) for p in p2_basis()])


def evaluate_p1(lam):
    return np.array([evaluate_poly(p, lam) for p in p1_basis()])


@lru_cache(maxsize=None)
def reference_integrals():
    """Geometry-free integrals (divided by 2|T|):
        Mr[m, n]       = int phi_m phi_n
        Kr[m, n, i, j] = int d_i phi_m d_j phi_n         (d_i = d/d lambda_i)
        Br[q, n, i]    = int psi_q d_i phi_n
        MPr[q, r]      = int psi_q psi_r
    """
    P2, P1 = p2_basis(), p1_basis()
    D = [[_d(p, i) for i in range(3)] for p in P2]
    Mr = np.array([[_int(_mul(a, b)) for b in P2] for a in P2])
    Kr = np.array([[[[_int(_mul(D[m][i], D[n][j])) for j in range(3)] for i in range(3)]
                    for n in range(6)] for m in range(6)])
    Br = np.array([[[_int(_mul(P1[q], D[n][i])) for i in range(3)] for n in range(6)] for q in range(3)])
    MPr = np.array([[_int(_mul(a, b)) for b in P1] for a in P1])
    return Mr, Kr, Br, MPr


def geometry(pts):
    """pts: (nt, 3, 2) physical vertex coordinates (counter-clockwise).
    Returns area (nt,) and grad lambda (nt, 3, 2)."""
    x, y = pts[..., 0], pts[..., 1]
    twoA = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    g = np.empty(pts.shape)
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        g[:, i, 0] = (y[:, j] - y[:, k]) / twoA
        g[:, i, 1] = (x[:, k] - x[:, j]) / twoA
    return 0.5 * twoA, g


def element_matrices(pts):
    """Exact element matrices on triangles pts (nt, 3, 2):
    K (nt,6,6), M (nt,6,6), Bx (nt,3,6), By (nt,3,6), MP (nt,3,3)."""
    Mr, Kr, Br, MPr = reference_integrals()
    area, g = geometry(pts)
    two = 2.0 * area
    G = np.einsum('tic,tjc->tij', g, g)
    K = two[:, None, None] * np.einsum('tij,mnij->tmn', G, Kr)
    M = two[:, None, None] * Mr[None]
    Bx = two[:, None, None] * np.einsum('ti,qni->tqn', g[:, :, 0], Br)
    By = two[:, None, None] * np.einsum('ti,qni->tqn', g[:, :, 1], Br)
    MP = two[:, None, None] * MPr[None]
    return K, M, Bx, By, MP


# ---------------------------------------------------------------- global assembly

class Discretization:
    """Assembled matrices of one grid level (Sec. 2, eq. gen:bil:mv) in canonical lattice order."""

    def __init__(self, m: meshmod.Mesh):
        self.mesh = m
        self.n = m.n
        n = m.n
        self.n2 = (2 * n + 1) ** 2
        self.nv = (n + 1) ** 2
        lat2 = meshmod.lattice_index(m.p2_coords, n)          # P2 node id -> lattice index
        assert len(lat2) == self.n2 and len(np.unique(lat2)) == self.n2
        latv = meshmod.vertex_lattice_index(m.verts, n)
        assert len(latv) == self.nv and len(np.unique(latv)) == self.nv
        pts = m.verts[m.tris].astype(np.float64) / (2 * n)     # physical coordinates
        K, M, Bx, By, MP = element_matrices(pts)
        rows2 = lat2[m.tri_p2]                                 # (nt, 6)
        rowsv = latv[m.tris]                                   # (nt, 3)
        self.K = _assemble(K, rows2, rows2, self.n2, self.n2)
        self.M = _assemble(M, rows2, rows2, self.n2, self.n2)
        self.Bx = _assemble(Bx, rowsv, rows2, self.nv, self.n2)
        self.By = _assemble(By, rowsv, rows2, self.nv, self.n2)
        self.MP = _assemble(MP, rowsv, rowsv, self.nv, self.nv)
        coords = np.zeros((self.n2, 2), dtype=np.int64)
        coords[lat2] = m.p2_coords
        self.coords = coords                                   # lattice coords by lattice index
        self.interior = np.flatnonzero(~meshmod.on_boundary(coords, n))
        self.ni = len(self.interior)
        I = self.interior
        self.Ki = self.K[I][:, I].tocsr()
        self.Mi = self.M[I][:, I].tocsr()
        self.Bi = sp.hstack([self.Bx[:, I], self.By[:, I]]).tocsr()   # (nv, 2 ni)
        self.w = np.asarray(self.MP.sum(axis=1)).ravel()             # w = M_P 1 = int psi_i
        self.pnodes = np.arange(self.nv)                             # pressure unknowns: every vertex

    # sizes of the unknown vector x = [u_x (ni); u_y (ni); p (nv)]
    @property
    def nu(self):
        return 2 * self.ni

    @property
    def ndof(self):
        return 2 * self.ni + self.nv

    def A(self, beta):
        a = (self.Ki + beta * self.Mi).tocsr()
        return sp.block_diag([a, a]).tocsr()

    def system(self, beta):
        """The saddle-point matrix [[A, B^T], [B, 0]] of eq. gen:bil:mv."""
        return sp.bmat([[self.A(beta), self.Bi.T], [self.Bi, None]]).tocsr()

    def mass_u(self):
        return sp.block_diag([self.Mi, self.Mi]).tocsr()

    # --------------------------------------------------------- lattice <-> unknown vector
    def to_vec(self, u, p):
        """u: (2, 2N+1, 2N+1) lattice array, p: (N+1, N+1) -> unknown vector."""
        u = np.asarray(u, dtype=np.float64).reshape(2, -1)
        return np.concatenate([u[0][self.interior], u[1][self.interior], np.asarray(p, np.float64).ravel()])

    def from_vec(self, x):
        n = self.n
        u = np.zeros((2, self.n2))
        u[0][self.interior] = x[:self.ni]
        u[1][self.interior] = x[self.ni:2 * self.ni]
        return u.reshape(2, 2 * n + 1, 2 * n + 1), x[2 * self.ni:].reshape(n + 1, n + 1).copy()

    # --------------------------------------------------------- load vectors (Sec. 1 data f, g)
    def load(self, f_nodal, g_nodal, project_g=False):
        """Load vector of f, g given by nodal values: f_vec = (f_h, phi_i) on interior P2 nodes,
        g_vec = (g_h, psi_i) on all vertices, where f_h, g_h interpolate the nodal values on the
        full lattice (boundary values included).  With project_g, the P1 function g_h is first
        shifted to zero mean, g_h <- g_h - (w^T g)/(w^T 1) (the solvability condition, Sec. 1)."""
        f_nodal = np.asarray(f_nodal, np.float64).reshape(2, -1)
        g_nodal = np.asarray(g_nodal, np.float64).ravel().copy()
        if project_g:
            g_nodal = g_nodal - (self.w @ g_nodal) / self.w.sum()
        fx = (self.M @ f_nodal[0])[self.interior]
        fy = (self.M @ f_nodal[1])[self.interior]
        g = self.MP @ g_nodal
        return np.concatenate([fx, fy, g])


def _assemble(E, rows, cols, nr, nc):
    nt, a, b = E.shape
    r = np.repeat(rows, b, axis=1).reshape(nt, a, b)
    c = np.tile(cols, (1, a)).reshape(nt, a, b)
    return sp.coo_matrix((E.ravel(), (r.ravel(), c.ravel())), shape=(nr, nc)).tocsr()


def discretizations(levels: int):
    return [Discretization(m) for m in meshmod.hierarchy(levels)]


# ---------------------------------------------------------------- error norms (for pins)

def _collapsed_gauss(npts):
    """Quadrature on the reference triangle {xi1, xi2 >= 0, xi1 + xi2 <= 1} from a Gauss-Legendre
    tensor rule through the collapsing map xi1 = s, xi2 = t (1 - s); exact for total degree
    <= 2*npts - 2.  Returns barycentric points (3, q) and weights summing to 1/2."""
    x, w = np.polynomial.legendre.leggauss(npts)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    S, T = np.meshgrid(x, x, indexing="ij")
    WS, WT = np.meshgrid(w, w, indexing="ij")
    xi1 = S.ravel()
    xi2 = (T * (1.0 - S)).ravel()
    wt = (WS * WT * (1.0 - S)).ravel()
    return np.stack([1.0 - xi1 - xi2, xi1, xi2]), wt


def error_norms(disc: "Discretization", u_lat, p_lat, exact_u, exact_grad_u, exact_p, npts=6):
    """L2 and H1-seminorm errors of the P2 velocity and L2 error of the P1 pressure against
    analytic functions, by quadrature over every triangle."""
    m = disc.mesh
    n = m.n
    lam, wq = _collapsed_gauss(npts)
    P2 = p2_basis()
    phi = np.stack([evaluate_poly(p, lam) for p in P2])                       # (6, q)
    dphi = np.stack([[evaluate_poly(_d(p, i), lam) * np.ones_like(lam[0]) for i in range(3)]
                     for p in P2])                                            # (6, 3, q)
    pts = m.verts[m.tris].astype(np.float64) / (2 * n)                        # (nt, 3, 2)
    area, g = geometry(pts)
    xq = np.einsum('iq,tic->tqc', lam, pts)                                   # (nt, q, 2)
    lat2 = lattice_index_of(m)
    latv = (m.verts[:, 1] // 2) * (n + 1) + m.verts[:, 0] // 2
    u = np.asarray(u_lat, np.float64).reshape(2, -1)
    pv = np.asarray(p_lat, np.float64).ravel()
    ue = exact_u(xq[..., 0], xq[..., 1])
    ge = exact_grad_u(xq[..., 0], xq[..., 1])
    pe = exact_p(xq[..., 0], xq[..., 1])
    W = 2.0 * area[:, None] * wq[None, :]
    l2u = h1u = 0.0
    for c in range(2):
        coef = u[c][lat2[m.tri_p2]]                                           # (nt, 6)
        uh = coef @ phi                                                       # (nt, q)
        l2u += np.sum(W * (uh - ue[c]) ** 2)
        # grad u_h = sum_a coef_a sum_i dphi_a/dlambda_i grad lambda_i
        gl = np.einsum('ta,aiq->tiq', coef, dphi)                              # (nt, 3, q)
        for d in range(2):
            gh = np.einsum('tiq,ti->tq', gl, g[:, :, d])
            h1u += np.sum(W * (gh - ge[c][d]) ** 2)
    ph = pv[latv[m.tris]] @ lam                                               # (nt, q)
    l2p = np.sum(W * (ph - pe) ** 2)
    return np.sqrt(l2u), np.sqrt(h1u), np.sqrt(l2p)


def lattice_index_of(m):
    return m.p2_coords[:, 1] * (2 * m.n + 1) + m.p2_coords[:, 0]
