"""The L-shaped domain: the unit square without its upper-right quadrant [1/2, 1]^2.

TEST INFRASTRUCTURE (part of the oracle package): only tests, the smoke check and the benchmark's
CPU baseline may import it.

Sec. 1: the convergence analysis uses regularity results that need a convex domain, but the method
itself applies to non-convex domains; the L-shape is the standard one.  The discretization is the
one of Sec. 2 on the triangles of the unit-square meshes (mesh.py) that lie in the L:
  * level j of the L-shaped hierarchy is level j + 1 of the square without the triangles in the
    removed quadrant (the square's level-0 fan has no vertex inside the L, and the Taylor-Hood
    pair needs interior vertices, Sec. 2);
  * velocity unknowns: the P2 nodes of the kept triangles that are not on the boundary of the L
    (the outer sides and the re-entrant sides x = 1/2, y >= 1/2 and y = 1/2, x >= 1/2);
  * pressure unknowns: the vertices of the kept triangles, with zero mean over the L.
Two triangles, at the convex corners (1, 1/2) and (1/2, 1), have all three vertices on the
boundary; B^T still has only the constant pressure in its kernel (tests/test_oracle_lshape.py), so
the problem with the zero-mean condition is well posed.  Lattice arrays keep the square's layout
((2N+1)^2 and (N+1)^2); entries outside the L are zero.
"""
from dataclasses import replace

import numpy as np
import scipy.sparse as sp

from . import fem
from . import mesh as meshmod


def _kept(m: meshmod.Mesh):
    """Triangles of the square mesh m inside the L (centroid outside the removed quadrant)."""
    c = m.verts[m.tris].sum(axis=1)                     # 3 x centroid, lattice units
    half3 = 3 * m.n                                     # 3 x (1/2) in lattice units of 1/(2N)
    return ~((c[:, 0] > half3) & (c[:, 1] > half3))


def hierarchy(levels: int):
    """L-shaped meshes for j = 0 .. levels-1 (square levels 1 .. levels): the kept triangles, their
    P2 node ids, and parents renumbered to the kept triangles of the next coarser L mesh."""
    sq = meshmod.hierarchy(levels + 1)
    out = []
    prev_new = None
    for lev in range(1, levels + 1):
        m = sq[lev]
        keep = _kept(m)
        idx = np.flatnonzero(keep)
        if prev_new is None:
            parent = -np.ones(len(idx), dtype=np.int64)
        else:
            parent = prev_new[m.parent[idx]]
            assert np.all(parent >= 0)                  # children of kept triangles only
        new = -np.ones(len(m.tris), dtype=np.int64)
        new[idx] = np.arange(len(idx))
        prev_new = new
        out.append(replace(m, level=lev - 1, tris=m.tris[idx], tri_p2=m.tri_p2[idx], parent=parent))
    return out


def on_boundary(coords, n):
    """P2-lattice coordinates on the boundary of the L (outer sides and re-entrant sides)."""
    X, Y = coords[:, 0], coords[:, 1]
    return (X == 0) | (Y == 0) | (X == 2 * n) | (Y == 2 * n) | ((X == n) & (Y >= n)) | ((Y == n) & (X >= n))


class LDiscretization(fem.Discretization):
    """The matrices of eq. gen:bil:mv on the L: assembled over the kept triangles only (so rows of
    nodes outside the L are zero), restricted to the L's unknowns."""

    def __init__(self, m: meshmod.Mesh):
        super().__init__(m)                             # assembles K, M, Bx, By, MP over m.tris
        n = m.n
        lat2 = meshmod.lattice_index(m.p2_coords, n)
        latv = meshmod.vertex_lattice_index(m.verts, n)
        used2 = np.unique(lat2[m.tri_p2])
        self.interior = np.intersect1d(used2, np.flatnonzero(~on_boundary(self.coords, n)))
        self.ni = len(self.interior)
        self.pnodes = np.unique(latv[m.tris])
        I, P = self.interior, self.pnodes
        self.Ki = self.K[I][:, I].tocsr()
        self.Mi = self.M[I][:, I].tocsr()
        self.Bi = sp.hstack([self.Bx[P][:, I], self.By[P][:, I]]).tocsr()
        self.MPfull = self.MP
        self.MP = self.MPfull[P][:, P].tocsr()
        self.w = np.asarray(self.MP.sum(axis=1)).ravel()

    @property
    def ndof(self):
        return 2 * self.ni + len(self.pnodes)

    def to_vec(self, u, p):
        u = np.asarray(u, dtype=np.float64).reshape(2, -1)
        p = np.asarray(p, np.float64).ravel()
        return np.concatenate([u[0][self.interior], u[1][self.interior], p[self.pnodes]])

    def from_vec(self, x):
        n = self.n
        u = np.zeros((2, self.n2))
        u[0][self.interior] = x[:self.ni]
        u[1][self.interior] = x[self.ni:2 * self.ni]
        p = np.zeros(self.nv)
        p[self.pnodes] = x[2 * self.ni:]
        return u.reshape(2, 2 * n + 1, 2 * n + 1), p.reshape(n + 1, n + 1)

    def load(self, f_nodal, g_nodal, project_g=False):
        """Load vectors of nodal data on the L: f = (f_h, phi_i) on the interior P2 nodes, g =
        (g_h, psi_i) on the L's vertices; with project_g, g_h is first shifted to zero mean on the L."""
        f_nodal = np.asarray(f_nodal, np.float64).reshape(2, -1)
        g = np.asarray(g_nodal, np.float64).ravel()[self.pnodes].copy()
        if project_g:
            g = g - (self.w @ g) / self.w.sum()
        fx = (self.M @ f_nodal[0])[self.interior]
        fy = (self.M @ f_nodal[1])[self.interior]
        return np.concatenate([fx, fy, self.MP @ g])


def discretizations(levels: int):
    return [LDiscretization(m) for m in hierarchy(levels)]
