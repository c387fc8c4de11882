"""Host logic of the CUDA library, checked without a GPU: the stencil class of every cell and the
node-stencil rows the kernels apply (C-ABI stokes_stencil_class, stokes_stencil_rows) against the
oracle's mesh and its assembled matrices of eq. gen:bil:mv; the canonical embedding weights of the
transfer kernels (stokes_transfer_weights) and of the coarse-grid correction compiled into the
planar smoothing kernel (stokes_embed_weights) against the oracle's prolongation; and the level-0
bordered inverse (stokes_coarse_inverse) against a dense inverse of the oracle's level-0 matrix.

The class of a cell is read here from the oracle's triangle list: the orientation of each of its
four squares is the direction of that square's diagonal edge ("/" = 0, "\\" = 1), and the four
bits (square (i, j), (i-1, j), (i, j-1), (i-1, j-1)) name the class (0x0 -> 0, 0xF -> 1, the
mid-line patterns 0x5, 0xA, 0x3, 0xC -> 2..5, the centre 0x6 -> 6)."""
import ctypes

import numpy as np
import pytest

from oracle import fem

PATTERN_TO_CLASS = {0x0: 0, 0xF: 1, 0x5: 2, 0xA: 3, 0x3: 4, 0xC: 5, 0x6: 6}


def square_orientations(m):
    """orient[a, b] of the square with lower-left vertex (a/N, b/N), from the diagonal edges."""
    n = m.n
    orient = -np.ones((n, n), dtype=int)
    P = m.verts[m.tris]                                   # P2-lattice coordinates, vertices even
    for e0, e1 in ((0, 1), (1, 2), (2, 0)):
        d = P[:, e1] - P[:, e0]
        diag = (np.abs(d[:, 0]) == 2) & (np.abs(d[:, 1]) == 2)
        lo = np.minimum(P[diag, e0], P[diag, e1]) // 2
        orient[lo[:, 0], lo[:, 1]] = np.where(d[diag, 0] * d[diag, 1] > 0, 0, 1)
    assert (orient >= 0).all()
    return orient


def cell_class(orient, i, j):
    bits = orient[i, j] | (orient[i - 1, j] << 1) | (orient[i, j - 1] << 2) | (orient[i - 1, j - 1] << 3)
    return PATTERN_TO_CLASS[int(bits)]


@pytest.fixture(scope="module")
def lib():
    from paper_1502_04070_gb300 import _binding
    return _binding.load()


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(5)


@pytest.mark.parametrize("k", [2, 4])
def test_stencil_classes_match_the_mesh(lib, discs, k):
    m = discs[k].mesh
    n = m.n
    orient = square_orientations(m)
    seen = set()
    out = ctypes.c_int()
    for i in range(1, n):
        for j in range(1, n):
            assert lib.stokes_stencil_class(k + 1, i, j, ctypes.byref(out)) == 0
            c = cell_class(orient, i, j)
            assert out.value == c, (i, j, out.value, c)
            seen.add(c)
    assert seen == set(range(7))


@pytest.mark.parametrize("beta", [0.0, 7.5, 1e6])
@pytest.mark.parametrize("k", [3, 4])
def test_stencil_rows_match_the_assembled_matrices(lib, discs, k, beta):
    d = discs[k]
    n = d.n
    A = (d.K + beta * d.M).tocsr()
    Bx, By = d.Bx.tocsr(), d.By.tocsr()
    BxT, ByT = Bx.T.tocsr(), By.T.tocsr()
    lat = lambda X, Y: Y * (2 * n + 1) + X
    vert = lambda a, b: b * (n + 1) + a
    orient = square_orientations(d.mesh)
    buf = {nm: np.zeros(sz) for nm, sz in (("ma", 100), ("mbtx", 36), ("mbty", 36), ("mbx", 25), ("mby", 25),
                                           ("midg", 4))}
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for cls in range(7):
        assert lib.stokes_stencil_rows(k + 1, float(beta), cls, *(ptr(buf[nm]) for nm in
                                       ("ma", "mbtx", "mbty", "mbx", "mby", "midg"))) == 0
        cells = [(i, j) for i in range(2, n - 1) for j in range(2, n - 1) if cell_class(orient, i, j) == cls]
        assert cells
        for (i, j) in cells[:6]:
            win = [(dx, dy) for dy in range(-2, 3) for dx in range(-2, 3)]
            vwin = [(di, dj) for dj in range(-1, 2) for di in range(-1, 2)]
            for s in range(4):
                X, Y = 2 * i + (s & 1), 2 * j + (s >> 1)
                row = A[lat(X, Y)].toarray().ravel()
                scale = np.abs(row).max()
                for w, (dx, dy) in enumerate(win):
                    c = lat(2 * i + dx, 2 * j + dy)
                    assert abs(buf["ma"][s * 25 + w] - row[c]) <= 1e-13 * scale, (cls, s, dx, dy)
                    row[c] = 0.0
                assert np.abs(row).max() == 0.0                       # no coupling outside the window
                assert abs(buf["midg"][s] * A[lat(X, Y), lat(X, Y)] - 1.0) <= 1e-14
                for name, BT in (("mbtx", BxT), ("mbty", ByT)):
                    col = BT[lat(X, Y)].toarray().ravel()
                    bscale = max(np.abs(col).max(), 1e-300)
                    for w, (di, dj) in enumerate(vwin):
                        v = vert(i + di, j + dj)
                        assert abs(buf[name][s * 9 + w] - col[v]) <= 1e-13 * bscale, (name, cls, s, di, dj)
                        col[v] = 0.0
                    assert np.abs(col).max() == 0.0
            for name, Bm in (("mbx", Bx), ("mby", By)):
                row = Bm[vert(i, j)].toarray().ravel()
                bscale = np.abs(row).max()
                for w, (dx, dy) in enumerate(win):
                    c = lat(2 * i + dx, 2 * j + dy)
                    assert abs(buf[name][w] - row[c]) <= 1e-13 * bscale, (name, cls, dx, dy)
                    row[c] = 0.0
                assert np.abs(row).max() == 0.0


def test_table_entry_points_reject_bad_arguments(lib):
    out = ctypes.c_int()
    a = np.zeros(100)
    p = a.ctypes.data_as(ctypes.c_void_p)
    assert lib.stokes_stencil_class(0, 1, 1, ctypes.byref(out)) != 0
    assert lib.stokes_stencil_class(3, -1, 1, ctypes.byref(out)) != 0
    assert lib.stokes_stencil_class(3, 1, 9, ctypes.byref(out)) != 0
    assert lib.stokes_stencil_rows(3, 1.0, 7, p, p, p, p, p, p) != 0
    assert lib.stokes_stencil_rows(3, -1.0, 0, p, p, p, p, p, p) != 0
    assert lib.stokes_stencil_rows(3, 1.0, 0, None, p, p, p, p, p) != 0


@pytest.mark.parametrize("levels", range(1, 14))
def test_register_tile_structure_holds_on_every_level(lib, levels):
    """The register-coefficient Uzawa tiles (step variants 10-11) hard-code which coefficients of the
    merged stencils of the two orientation classes vanish, which are equal (eight values for the
    42 nonzero A terms of a cell), and that every B and B^T entry is +-b or +-b/2.  The host check of
    that structure against the stencils the library builds (the rows pinned to the oracle's
    assembled matrices above) passes for every level and for beta from 0 to 1e12."""
    for beta in (0.0, 1e-3, 1.0, 37.0, 1e4, 1e8, 1e12):
        assert lib.stokes_step_tables_match(levels, beta) == 0, (levels, beta)
    assert lib.stokes_step_tables_match(0, 1.0) != 0
    assert lib.stokes_step_tables_match(3, -1.0) != 0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_fused_correction_table_equals_the_oracle_embedding(lib, discs, k):
    """The embedding weights compiled into the planar smoothing kernel for the coarse-grid
    correction it adds to its tiles (stokes_embed_weights, evaluated at compile time from the P2
    basis) equal the oracle's prolongation at the 16 fine lattice points each coarse square owns."""
    from oracle import transfer
    w = np.zeros(2 * 9 * 4 * 4)
    assert lib.stokes_embed_weights(w.ctypes.data_as(ctypes.c_void_p)) == 0
    w = w.reshape(2, 9, 4, 4)
    coarse, fine = discs[k], discs[k + 1]
    P2 = transfer.prolongation_full(coarse, fine)[0].toarray()
    nc, nf = coarse.n, fine.n
    orient = square_orientations(coarse.mesh)
    for a in range(nc):
        for b in range(nc):
            o = orient[a, b]
            for L in range(9):
                cc = (2 * b + L // 3) * (2 * nc + 1) + 2 * a + L % 3
                for fb in range(4):
                    for fa in range(4):
                        ff = (4 * b + fb) * (2 * nf + 1) + 4 * a + fa
                        assert abs(P2[ff, cc] - w[o, L, fb, fa]) <= 1e-14, (a, b, L, fa, fb)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_transfer_weights_equal_the_oracle_embedding(lib, discs, k):
    """The embedding weights the transfer kernels apply (stokes_transfer_weights) equal the oracle's
    prolongation (coarse basis functions evaluated at the fine nodes, Sec. 3) for every coarse
    square, local node and fine lattice point of the square."""
    from oracle import transfer
    w = np.zeros(2 * 9 * 5 * 5)
    assert lib.stokes_transfer_weights(w.ctypes.data_as(ctypes.c_void_p)) == 0
    w = w.reshape(2, 9, 5, 5)
    coarse, fine = discs[k], discs[k + 1]
    P2, _ = transfer.prolongation_full(coarse, fine)
    P2 = P2.toarray()
    nc, nf = coarse.n, fine.n
    orient = square_orientations(coarse.mesh)
    for a in range(nc):
        for b in range(nc):
            o = orient[a, b]
            for L in range(9):
                cc = (2 * b + L // 3) * (2 * nc + 1) + 2 * a + L % 3
                for fb in range(5):
                    for fa in range(5):
                        ff = (4 * b + fb) * (2 * nf + 1) + 4 * a + fa
                        assert abs(P2[ff, cc] - w[o, L, fb, fa]) <= 1e-14, (a, b, L, fa, fb)


@pytest.mark.parametrize("beta", [0.0, 1.0, 1e4])
def test_coarse_inverse_equals_the_oracle_bordered_solve(lib, discs, beta):
    """The level-0 inverse (host Gauss-Jordan, stokes_coarse_inverse) against a dense inverse of the
    oracle's bordered level-0 matrix; the unknown orders coincide (interior u_x, u_y row-major,
    then the vertex pressures)."""
    from oracle import multigrid as mg
    inv = np.zeros(27 * 27)
    assert lib.stokes_coarse_inverse(float(beta), inv.ctypes.data_as(ctypes.c_void_p)) == 0
    inv = inv.reshape(27, 27)
    H = mg.Hierarchy(1, beta, discs[:1])
    ref = np.linalg.inv(H.coarse_bordered)[:27, :27]
    assert np.abs(inv - ref).max() <= 1e-10 * np.abs(ref).max()
    assert lib.stokes_coarse_inverse(-1.0, inv.ctypes.data_as(ctypes.c_void_p)) != 0


@pytest.mark.parametrize("j", [1, 2, 3])
def test_lshape_reentrant_vertex_rows_equal_the_oracle(lib, j):
    """L-shaped domain: the B rows and pressure-mass weights of the vertices on the re-entrant sides
    (stokes_lshape_vertex_rows, summed over the squares inside the L) equal the rows of the
    oracle's masked assembly (oracle/lshape.py) at every such vertex of L-level j."""
    from oracle import lshape
    d = lshape.discretizations(j + 1)[j]
    n = d.n
    levels = j + 2                                     # L-level j is the square's level j + 1
    assert 2 ** levels == n
    Bx, By = d.Bx.tocsr(), d.By.tocsr()
    wfull = np.asarray(d.MPfull.sum(axis=1)).ravel()
    lat = lambda X, Y: Y * (2 * n + 1) + X
    h = n // 2
    verts = {0: [(h, y) for y in range(h + 1, n)], 1: [(x, h) for x in range(h + 1, n)], 2: [(h, h)],
             3: [(h, n)], 4: [(n, h)]}
    mbx, mby, w = np.zeros(25), np.zeros(25), ctypes.c_double()
    for kind, vs in verts.items():
        assert lib.stokes_lshape_vertex_rows(levels, kind, mbx.ctypes.data_as(ctypes.c_void_p),
                                             mby.ctypes.data_as(ctypes.c_void_p), ctypes.byref(w)) == 0
        for (i, jj) in vs:
            v = jj * (n + 1) + i
            assert abs(w.value - wfull[v]) <= 1e-15, (kind, i, jj)
            for name, Bm, tab in (("x", Bx, mbx), ("y", By, mby)):
                row = Bm[v].toarray().ravel()
                scale = np.abs(row).max()
                for dy in range(-2, 3):
                    for dx in range(-2, 3):
                        X, Y = 2 * i + dx, 2 * jj + dy
                        if 0 <= X <= 2 * n and 0 <= Y <= 2 * n:
                            c = lat(X, Y)
                            assert abs(tab[(dy + 2) * 5 + dx + 2] - row[c]) <= 1e-13 * scale, (kind, name, dx, dy)
                            row[c] = 0.0
                assert np.abs(row).max() == 0.0
    assert lib.stokes_lshape_vertex_rows(1, 0, mbx.ctypes.data_as(ctypes.c_void_p),
                                         mby.ctypes.data_as(ctypes.c_void_p), ctypes.byref(w)) != 0


@pytest.mark.parametrize("beta", [0.0, 10.0, 1e6])
@pytest.mark.parametrize("j", [1, 3])
def test_lshape_reentrant_schur_diagonal_equals_the_oracle(lib, j, beta):
    """L-shaped domain: S_hat = diag(B Ahat^-1 B^T) at the re-entrant vertices (stokes_lshape_schur)
    equals the oracle's S_hat on the L (multigrid.Level over the masked discretization), including
    the vertices next to the outer boundary where fewer velocity unknowns remain."""
    from oracle import lshape
    from oracle import multigrid as mg
    ds = lshape.discretizations(j + 1)
    d = ds[j]
    n = d.n
    H = mg.Hierarchy(j + 1, beta, ds)
    shat = H.levels[j].Shat
    pos = {int(v): k for k, v in enumerate(d.pnodes)}
    h = n // 2
    s0, s1, s2 = np.zeros(h), np.zeros(h), np.zeros(1)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.stokes_lshape_schur(j + 2, float(beta), ptr(s0), ptr(s1), ptr(s2)) == 0
    for t in range(h):                                 # t = h - 1: the ends on the outer boundary
        for got, (i, jj) in ((s0[t], (h, h + 1 + t)), (s1[t], (h + 1 + t, h))):
            ref = shat[pos[jj * (n + 1) + i]]
            assert abs(got - ref) <= 1e-12 * ref, (t, i, jj, got, ref)
    ref = shat[pos[h * (n + 1) + h]]
    assert abs(s2[0] - ref) <= 1e-12 * ref


@pytest.mark.parametrize("beta", [0.0, 1.0, 1e4])
def test_lshape_coarse_inverse_equals_the_oracle(lib, beta):
    """Level 0 of the L-shaped hierarchy: the host inverse (stokes_lshape_coarse_inverse) against a
    dense inverse of the oracle's bordered level-0 matrix on the L (same unknown order)."""
    from oracle import lshape
    from oracle import multigrid as mg
    d0 = lshape.discretizations(1)[0]
    inv = np.zeros(87 * 87)
    nunk = ctypes.c_int()
    assert lib.stokes_lshape_coarse_inverse(float(beta), inv.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nunk)) == 0
    assert nunk.value == d0.ndof == 87
    H = mg.Hierarchy(1, beta, [d0])
    ref = np.linalg.inv(H.coarse_bordered)[:87, :87]
    assert np.abs(inv.reshape(87, 87) - ref).max() <= 1e-10 * np.abs(ref).max()
