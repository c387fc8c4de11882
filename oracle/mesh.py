"""Mesh hierarchy of the numerical experiments (Sec. 6): unit square, 8 coarse triangles, red refinement.

Reading of the missing figure (Sec. 6, Fig. 1): the coarsest mesh is the fan of 8 triangles
around the centre (1/2, 1/2) over the 3x3 vertex grid {0, 1/2, 1}^2.  It is the only split of
that grid into 8 triangles in which every triangle has a vertex inside the domain (the centre),
which the inf-sup condition of the Taylor-Hood pair requires (Sec. 2, after eq. cond:s).

Each refinement step splits every triangle into four through its edge midpoints (Sec. 6).
The mesh is built explicitly as a triangle list; no lattice formula is used to produce it.

Coordinates are exact integers: on level k the P2 node lattice has spacing 1/(2N), N = 2^(k+1),
and every vertex and edge midpoint sits at integer coordinates (X, Y) in [0, 2N]^2.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    level: int
    n: int                      # N = 2^(level+1): number of element legs per side
    verts: np.ndarray           # (nv, 2) int, P2-lattice coordinates (multiples of 2)
    tris: np.ndarray            # (nt, 3) int, counter-clockwise vertex indices
    parent: np.ndarray          # (nt,) int, index of the parent triangle on level-1 (-1 on level 0)
    # P2 data (filled by build_p2)
    p2_coords: np.ndarray = field(default=None)   # (n2, 2) int lattice coords of P2 nodes
    tri_p2: np.ndarray = field(default=None)      # (nt, 6) P2 node ids: v0, v1, v2, m12, m02, m01


def coarse_mesh() -> Mesh:
    """Level 0: fan of 8 triangles around the centre of the 3x3 vertex grid (Sec. 6)."""
    # P2 lattice of level 0 has spacing 1/4: vertex grid {0, 1/2, 1} -> {0, 2, 4}
    verts = np.array([(2 * x, 2 * y) for y in range(3) for x in range(3)], dtype=np.int64)
    centre = 4
    ring = [(0, 0), (1, 0), (2, 0), (2, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    ring_ids = [y * 3 + x for (x, y) in ring]
    tris = []
    for a in range(8):
        b = (a + 1) % 8
        tris.append((centre, ring_ids[a], ring_ids[b]))
    tris = np.array(tris, dtype=np.int64)
    m = Mesh(level=0, n=2, verts=verts, tris=tris, parent=-np.ones(len(tris), dtype=np.int64))
    _orient_ccw(m)
    return m


def _orient_ccw(m: Mesh) -> None:
    p = m.verts[m.tris]
    d = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])
    assert np.all(d != 0)
    flip = d < 0
    m.tris[flip] = m.tris[flip][:, [0, 2, 1]]


def refine(m: Mesh) -> Mesh:
    """Red refinement: every triangle is split into 4 by joining its edge midpoints (Sec. 6)."""
    verts = [tuple(2 * v) for v in m.verts]          # lattice spacing halves: coordinates double
    index = {v: i for i, v in enumerate(verts)}

    def mid(i, j):
        a, b = verts[i], verts[j]
        c = ((a[0] + b[0]) // 2, (a[1] + b[1]) // 2)
        if c not in index:
            index[c] = len(verts)
            verts.append(c)
        return index[c]

    tris, parent = [], []
    for t, (a, b, c) in enumerate(m.tris):
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        for tri in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)):
            tris.append(tri)
            parent.append(t)
    out = Mesh(level=m.level + 1, n=2 * m.n, verts=np.array(verts, dtype=np.int64),
               tris=np.array(tris, dtype=np.int64), parent=np.array(parent, dtype=np.int64))
    _orient_ccw(out)
    return out


def build_p2(m: Mesh) -> Mesh:
    """P2 nodes = vertices + edge midpoints; returns the mesh with P2 node data filled in."""
    coords = [tuple(v) for v in m.verts]
    index = {v: i for i, v in enumerate(coords)}
    tri_p2 = np.zeros((len(m.tris), 6), dtype=np.int64)
    for t, (a, b, c) in enumerate(m.tris):
        ids = [a, b, c]
        for (i, j) in ((b, c), (a, c), (a, b)):
            pi, pj = coords[i], coords[j]
            q = ((pi[0] + pj[0]) // 2, (pi[1] + pj[1]) // 2)
            if q not in index:
                index[q] = len(coords)
                coords.append(q)
            ids.append(index[q])
        tri_p2[t] = ids
    m.p2_coords = np.array(coords, dtype=np.int64)
    m.tri_p2 = tri_p2
    return m


def hierarchy(levels: int):
    """Meshes for k = 0 .. levels-1, each with its P2 node data."""
    out = [build_p2(coarse_mesh())]
    for _ in range(1, levels):
        nxt = refine(out[-1])
        # P2 coordinates of the coarse mesh double on the finer lattice only through refine()
        out.append(build_p2(nxt))
    return out


def lattice_index(coords: np.ndarray, n: int) -> np.ndarray:
    """Flat index of P2-lattice coordinates (X, Y) in the canonical (2N+1)^2 row-major array
    (y outer, x inner)."""
    return coords[:, 1] * (2 * n + 1) + coords[:, 0]


def vertex_lattice_index(coords: np.ndarray, n: int) -> np.ndarray:
    """Flat index of a vertex (even P2-lattice coordinates) in the canonical (N+1)^2 pressure array."""
    assert np.all(coords % 2 == 0)
    return (coords[:, 1] // 2) * (n + 1) + coords[:, 0] // 2


def on_boundary(coords: np.ndarray, n: int) -> np.ndarray:
    return (coords[:, 0] == 0) | (coords[:, 1] == 0) | (coords[:, 0] == 2 * n) | (coords[:, 1] == 2 * n)
