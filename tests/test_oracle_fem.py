"""Pins of the oracle's discretisation against closed forms, symbolic integration and invariants.

Nothing here re-types the oracle's own formulas: element matrices are compared with sympy's
symbolic integrals of a Lagrange basis built by solving interpolation conditions, the monomial
rule with numerical quadrature, the appendix constants with their closed forms, and global
matrices with identities that hold for any correct assembly.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import fem, mesh, transfer


def test_monomial_rule_vs_numerical_quadrature():
    # reference triangle (0,0),(1,0),(0,1): lambda = (1-x-y, x, y), |T| = 1/2
    for e in [(0, 0, 0), (1, 0, 0), (2, 1, 0), (1, 1, 1), (0, 3, 1), (2, 2, 0), (4, 0, 0)]:
        f = lambda y, x: (1 - x - y) ** e[0] * x ** e[1] * y ** e[2]
        val, _ = scipy.integrate.dblquad(f, 0, 1, 0, lambda x: 1 - x, epsabs=1e-13, epsrel=1e-13)
        assert abs(val - 2 * 0.5 * fem.monomial_integral_over_2area(e)) < 1e-12


def test_appendix_constants():
    """Appendix (proof of the inverse inequality): on the reference element, with psi = 1 - xi_2
    (case 1) or psi = xi_2 (case 2), (p, p) <= C (p, psi p) for linear p holds with
    C = (6 + sqrt 6)/3 and C = 4 + sqrt 6; C is the largest generalized eigenvalue."""
    # barycentric on (0,0),(1,0),(0,1): lambda_0 = 1-xi1-xi2, lambda_1 = xi1, lambda_2 = xi2
    P1 = fem.p1_basis()
    M = np.array([[fem._int(fem._mul(a, b)) for b in P1] for a in P1])
    psi1 = {(1, 0, 0): 1.0, (0, 1, 0): 1.0}      # 1 - xi2 = lambda_0 + lambda_1
    psi2 = {(0, 0, 1): 1.0}                      # xi2 = lambda_2
    for psi, C in ((psi1, (6 + math.sqrt(6)) / 3), (psi2, 4 + math.sqrt(6))):
        Mpsi = np.array([[fem._int(fem._mul(fem._mul(a, b), psi)) for b in P1] for a in P1])
        lam = scipy.linalg.eigh(M, Mpsi, eigvals_only=True)
        assert abs(lam.max() - C) < 1e-12


def _sympy_element(pts):
    sympy = pytest.importorskip("sympy")
    x, y, s, t = sympy.symbols("x y s t")
    P = [sympy.Rational(*p) if isinstance(p, tuple) else p for p in pts]
    v = [sympy.Matrix(p) for p in pts]
    nodes = [v[0], v[1], v[2], (v[1] + v[2]) / 2, (v[0] + v[2]) / 2, (v[0] + v[1]) / 2]
    mono = [1, x, y, x * x, x * y, y * y]
    V = sympy.Matrix([[sympy.sympify(m).subs({x: nd[0], y: nd[1]}) for m in mono] for nd in nodes])
    C = V.inv()                                    # columns: coefficients of Lagrange basis
    phi = [sum(C[j, a] * mono[j] for j in range(6)) for a in range(6)]
    Vl = sympy.Matrix([[1, v[a][0], v[a][1]] for a in range(3)])
    Cl = Vl.inv()
    psi = [Cl[0, a] + Cl[1, a] * x + Cl[2, a] * y for a in range(3)]
    X = v[0] + s * (v[1] - v[0]) + t * (v[2] - v[0])
    J = abs((v[1] - v[0]).row_join(v[2] - v[0]).det())

    def integ(expr):
        e = sympy.expand(expr.subs({x: X[0], y: X[1]}, simultaneous=True))
        return sympy.integrate(sympy.integrate(e, (t, 0, 1 - s)), (s, 0, 1)) * J

    K = np.array([[float(integ(sympy.diff(phi[a], x) * sympy.diff(phi[b], x) + sympy.diff(phi[a], y) * sympy.diff(phi[b], y)))
                   for b in range(6)] for a in range(6)])
    M = np.array([[float(integ(phi[a] * phi[b])) for b in range(6)] for a in range(6)])
    Bx = np.array([[float(integ(sympy.diff(phi[b], x) * psi[q])) for b in range(6)] for q in range(3)])
    By = np.array([[float(integ(sympy.diff(phi[b], y) * psi[q])) for b in range(6)] for q in range(3)])
    return K, M, Bx, By


def test_element_matrices_vs_sympy():
    sympy = pytest.importorskip("sympy")
    R = sympy.Rational
    pts = [(R(1, 10), R(1, 5)), (R(7, 8), R(1, 3)), (R(2, 5), R(9, 10))]
    K, M, Bx, By = _sympy_element(pts)
    fp = np.array([[float(a) for a in p] for p in pts])[None]
    K2, M2, Bx2, By2, _ = fem.element_matrices(fp)
    for a, b in ((K, K2[0]), (M, M2[0]), (Bx, Bx2[0]), (By, By2[0])):
        assert np.abs(a - b).max() < 1e-13 * max(1.0, np.abs(a).max())


@pytest.fixture(scope="module")
def discs():
    return fem.discretizations(4)


def test_mesh_structure(discs):
    for k, d in enumerate(discs):
        n = 2 ** (k + 1)
        assert d.n == n and len(d.mesh.tris) == 8 * 4 ** k
        # every triangle has a vertex off the boundary (inf-sup condition of Sec. 2)
        v = d.mesh.verts[d.mesh.tris]
        inner = ~((v == 0) | (v == 2 * n)).any(axis=2)
        assert inner.any(axis=1).all()
    # level 0: the centre is a vertex of all 8 triangles
    assert np.all((discs[0].mesh.tris == 4).any(axis=1))


def test_global_invariants(discs):
    for d in discs:
        ones2 = np.ones(d.n2)
        assert np.abs(d.K @ ones2).max() < 1e-12                # stiffness kills constants
        assert abs(ones2 @ d.M @ ones2 - 1.0) < 1e-13           # |Omega| = 1
        assert abs(d.w.sum() - 1.0) < 1e-13
        assert abs(abs(d.K - d.K.T).max()) < 1e-14
        S = d.system(3.0)
        assert abs(S - S.T).max() < 1e-14
        assert np.abs(np.ones(d.nv) @ d.Bi).max() < 1e-13       # constants are in ker B^T
        assert d.ndof == 2 * (2 * d.n - 1) ** 2 + (d.n + 1) ** 2


def test_divergence_exact_for_quadratics(discs):
    """For a quadratic field v (P2-interpolated exactly), full B v = (div v, psi_i) computed with
    independent exact integration of the linear function div v against psi_i (via M_P, exact for
    P1 x P1)."""
    d = discs[-1]
    X = d.coords[:, 0] / (2 * d.n)
    Y = d.coords[:, 1] / (2 * d.n)
    vx = 1 + 2 * X - 3 * Y + X * X - 2 * X * Y + 0.5 * Y * Y
    vy = -1 + X + 4 * Y + 3 * X * Y - Y * Y + 2 * X * X
    divv = lambda x, y: (2 + 2 * x - 2 * y) + (4 + 3 * x - 2 * y)
    Bv = d.Bx @ vx + d.By @ vy
    vv = d.coords[(d.coords[:, 0] % 2 == 0) & (d.coords[:, 1] % 2 == 0)]
    order = np.argsort(mesh.vertex_lattice_index(vv, d.n))
    vv = vv[order] / (2 * d.n)
    ref = d.MP @ divv(vv[:, 0], vv[:, 1])
    assert np.abs(Bv - ref).max() < 1e-13


def test_prolongation_reproduces_polynomials(discs):
    for l in range(1, len(discs)):
        c, f = discs[l - 1], discs[l]
        P2, P1 = transfer.prolongation_full(c, f)
        q = lambda X, Y: 0.3 + X - 2 * Y + 3 * X * X - X * Y + 2 * Y * Y
        cx, cy = c.coords[:, 0] / (2 * c.n), c.coords[:, 1] / (2 * c.n)
        fx, fy = f.coords[:, 0] / (2 * f.n), f.coords[:, 1] / (2 * f.n)
        assert np.abs(P2 @ q(cx, cy) - q(fx, fy)).max() < 1e-13
        lin = lambda X, Y: 0.7 - 3 * X + 5 * Y
        cv = np.array([(i, j) for j in range(c.n + 1) for i in range(c.n + 1)]) / c.n
        fv = np.array([(i, j) for j in range(f.n + 1) for i in range(f.n + 1)]) / f.n
        assert np.abs(P1 @ lin(cv[:, 0], cv[:, 1]) - lin(fv[:, 0], fv[:, 1])).max() < 1e-13


@pytest.mark.parametrize("beta", [0.0, 1.0, 1e4])
def test_galerkin_identity(discs, beta):
    """Nested conforming spaces with exact integration: I^T A_k I = A_{k-1} (Sec. 2 nesting,
    Sec. 3 canonical transfers)."""
    for l in range(1, len(discs)):
        P = transfer.prolongation(discs[l - 1], discs[l])
        Sc = discs[l - 1].system(beta)
        Sf = discs[l].system(beta)
        G = (P.T @ Sf @ P).toarray()
        assert np.abs(G - Sc.toarray()).max() < 1e-12 * max(1.0, beta)
