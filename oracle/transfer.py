"""Canonical grid transfers between nested levels (Sec. 3).

The prolongation I_{k-1}^k is the canonical embedding of X_{k-1} into X_k: a coarse function is
written in the fine nodal basis by evaluating it at the fine nodes.  It is built here by direct
evaluation of every coarse basis function at the fine nodes of each child triangle (red refinement
keeps every fine triangle inside one coarse triangle).  The restriction I_k^{k-1} is its transpose.
Rows and columns of Dirichlet velocity nodes are dropped (both spaces are subspaces of H^1_0).
"""
import numpy as np
import scipy.sparse as sp

from . import fem


def _barycentric(tri_pts, q):
    """Barycentric coordinates of points q (n, 2) in triangles tri_pts (n, 3, 2)."""
    a, b, c = tri_pts[:, 0], tri_pts[:, 1], tri_pts[:, 2]
    v0, v1, v2 = b - a, c - a, q - a
    det = v0[:, 0] * v1[:, 1] - v0[:, 1] * v1[:, 0]
    l1 = (v2[:, 0] * v1[:, 1] - v2[:, 1] * v1[:, 0]) / det
    l2 = (v0[:, 0] * v2[:, 1] - v0[:, 1] * v2[:, 0]) / det
    return np.stack([1.0 - l1 - l2, l1, l2], axis=1)


def _dedup_coo(rows, cols, vals, shape):
    """Sparse matrix from (row, col, value) triples in which repeated pairs carry equal values
    (a fine node shared by several child triangles); each pair is kept once, zeros dropped."""
    keep = np.abs(vals) > 0
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    key = rows.astype(np.int64) * shape[1] + cols
    _, first = np.unique(key, return_index=True)
    return sp.coo_matrix((vals[first], (rows[first], cols[first])), shape=shape).tocsr()


def prolongation_full(coarse: fem.Discretization, fine: fem.Discretization):
    """Scalar P2 (n2_f x n2_c) and P1 (nv_f x nv_c) embeddings on the full lattices."""
    mc, mf = coarse.mesh, fine.mesh
    lat2c = mc.p2_coords[:, 1] * (2 * mc.n + 1) + mc.p2_coords[:, 0]
    lat2f = mf.p2_coords[:, 1] * (2 * mf.n + 1) + mf.p2_coords[:, 0]
    latvc = (mc.verts[:, 1] // 2) * (mc.n + 1) + mc.verts[:, 0] // 2
    latvf = (mf.verts[:, 1] // 2) * (mf.n + 1) + mf.verts[:, 0] // 2
    cverts = mc.verts.astype(np.float64) / (2 * mc.n)
    nt = len(mf.tris)
    T = mf.parent                                              # parent coarse triangle of each fine one
    # P2: every fine P2 node of every child, in its parent's barycentric coordinates
    tri = np.repeat(cverts[mc.tris[T]], 6, axis=0)             # (nt*6, 3, 2)
    fnodes = mf.p2_coords[mf.tri_p2].reshape(-1, 2).astype(np.float64) / (2 * mf.n)
    lam = _barycentric(tri, fnodes).T                          # (3, nt*6)
    vals = np.stack([fem.evaluate_poly(p, lam) for p in fem.p2_basis()], axis=1)   # (nt*6, 6)
    rows = np.repeat(lat2f[mf.tri_p2].reshape(-1), 6)
    cols = np.repeat(lat2c[mc.tri_p2[T]], 6, axis=0).reshape(-1)
    P2 = _dedup_coo(rows, cols, vals.reshape(-1), (fine.n2, coarse.n2))
    # P1: fine vertices (local nodes 0..2) in the parent's barycentric coordinates
    tri = np.repeat(cverts[mc.tris[T]], 3, axis=0)
    fv = mf.verts[mf.tris].reshape(-1, 2).astype(np.float64) / (2 * mf.n)
    lam = _barycentric(tri, fv).T
    vals = np.stack([fem.evaluate_poly(p, lam) for p in fem.p1_basis()], axis=1)  # (nt*3, 3)
    rows = np.repeat(latvf[mf.tris].reshape(-1), 3)
    cols = np.repeat(latvc[mc.tris[T]], 3, axis=0).reshape(-1)
    P1 = _dedup_coo(rows, cols, vals.reshape(-1), (fine.nv, coarse.nv))
    return P2, P1


def prolongation(coarse: fem.Discretization, fine: fem.Discretization):
    """I_{k-1}^k on the unknown vectors [u_x; u_y; p] (Dirichlet rows/columns dropped)."""
    P2, P1 = prolongation_full(coarse, fine)
    P2i = P2[fine.interior][:, coarse.interior]
    P1p = P1[fine.pnodes][:, coarse.pnodes]                    # pressure unknowns (all vertices on the square)
    return sp.block_diag([P2i, P2i, P1p]).tocsr()
