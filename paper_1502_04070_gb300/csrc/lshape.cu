// lshape.cu -- host tables for the L-shaped domain (the unit square without [1/2, 1]^2).
//
// Sec. 1: the convergence theory needs a convex domain, the method does not.  On the L the square's
// lattice and node stencils carry over unchanged at every velocity node strictly inside the L (all
// of its triangles lie in the L); the nodes on the re-entrant sides x = 1/2 (y >= 1/2) and
// y = 1/2 (x >= 1/2) join the Dirichlet set.  The pressure vertices on those sides stay unknowns,
// and their B rows and pressure-mass weights sum over the squares around the vertex that lie in
// the L only: this file computes those rows from the same square matrices as the square's tables.
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/stokes_mg.h"
#include "common.cuh"
#include "elements.h"

using namespace smg;

namespace {

// Squares around vertex (i, j): SQ 0 = (i, j), 1 = (i-1, j), 2 = (i, j-1), 3 = (i-1, j-1); the vertex
// is corner SQ of square SQ.  Squares in the removed quadrant, per kind of re-entrant vertex:
//   kind 0, side x = 1/2 above the corner: SQ 0 and 2 (to the right);
//   kind 1, side y = 1/2 right of the corner: SQ 0 and 1 (above);
//   kind 2, the corner (1/2, 1/2): SQ 0;
//   kind 3, the end (1/2, 1) of the side x = 1/2 on the outer boundary: SQ 0, 1 (outside) and 2;
//   kind 4, the end (1, 1/2) of the side y = 1/2 on the outer boundary: SQ 0, 2 (outside) and 1.
// The stencil classes of these cells (the mid-line cells above / right of the centre, and the
// centre cell) give the orientation of every square.
constexpr int kKinds = 5;
constexpr unsigned kRemoved[kKinds] = {0x5u, 0x3u, 0x1u, 0x7u, 0x7u};
constexpr int kClass[kKinds] = {3, 5, 6, 3, 5};

// Velocity lattice node (X, Y) of the P2 lattice ([0, 2n]^2) strictly inside the L: off the outer
// boundary and off the closed removed quadrant (whose edges are the re-entrant sides).
bool l_interior(int X, int Y, int n) {
    if (X <= 0 || Y <= 0 || X >= 2 * n || Y >= 2 * n) return false;
    return !(X >= n && Y >= n);
}

// Diagonal of A = K + beta M at an interior lattice node: the sum over the squares that contain it
// (orientation 0 in the lower-left and upper-right quadrants, 1 in the other two, Sec. 6 mesh).
double a_diag(const SquareMatrices& S, int X, int Y, int n, double beta) {
    const double h = 1.0 / n;
    double s = 0.0;
    for (int a = X / 2 - 1; a <= X / 2; ++a)
        for (int b = Y / 2 - 1; b <= Y / 2; ++b) {
            if (a < 0 || b < 0 || a >= n || b >= n || X < 2 * a || X > 2 * a + 2 || Y < 2 * b || Y > 2 * b + 2) continue;
            const int o = ((a < n / 2) != (b < n / 2)) ? 1 : 0;
            const int l = (Y - 2 * b) * 3 + (X - 2 * a);
            s += S.K[o][l][l] + beta * h * h * S.M[o][l][l];
        }
    return s;
}

// B row of a re-entrant vertex (kind as below) over its 5 x 5 lattice window, and its weight.
void vertex_rows(const SquareMatrices& S, int n, int kind, double* mbx, double* mby, double* w) {
    const double h = 1.0 / n;
    std::memset(mbx, 0, 25 * sizeof(double));
    std::memset(mby, 0, 25 * sizeof(double));
    *w = 0.0;
    for (int SQ = 0; SQ < 4; ++SQ) {
        if ((kRemoved[kind] >> SQ) & 1u) continue;
        const int o = sq_orient(kClass[kind], SQ);
        const int ox = -2 * (SQ & 1), oy = -2 * (SQ >> 1);      // square origin relative to (2i, 2j)
        for (int m = 0; m < 9; ++m) {
            const int dx = ox + m % 3, dy = oy + m / 3;
            mbx[(dy + 2) * 5 + dx + 2] += h * S.Bx[o][SQ][m];
            mby[(dy + 2) * 5 + dx + 2] += h * S.By[o][SQ][m];
        }
        for (int r = 0; r < 4; ++r) *w += h * h * S.MP[o][SQ][r];
    }
}

const SquareMatrices& squares_l() {
    static const SquareMatrices S = square_matrices();
    return S;
}

}  // namespace

namespace smg {

// Level 0 of the L-shaped hierarchy (the square's level with N = 4 without the upper-right quadrant)
// in the square's unknown order of bordered_system (size bordered_size(4) = 124): the system of
// eq. gen:bil:mv over the 12 squares of the L, the L's pressure weights in the border, and identity
// rows and columns at the square's unknowns that are not the L's (velocity nodes on the re-entrant
// sides or in the removed quadrant, vertices strictly inside it), so that the solution is zero there
// when the right-hand side is.
void lshape_bordered_system(double beta, double* M) {
    const SquareMatrices& S = squares_l();
    const int n = 4, nm = 2 * n - 1, nv = nm * nm, nb = bordered_size(n);
    const double h = 1.0 / n;
    std::memset(M, 0, sizeof(double) * (size_t)nb * nb);
    auto at = [&](int r, int c) -> double& { return M[(size_t)r * nb + c]; };
    auto vidx = [&](int c, int X, int Y) -> int {
        if (!l_interior(X, Y, n)) return -1;
        return c * nv + (Y - 1) * nm + (X - 1);
    };
    auto pidx = [&](int x, int y) { return 2 * nv + y * (n + 1) + x; };
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            if (a >= n / 2 && b >= n / 2) continue;                    // the removed quadrant
            const int o = ((a < n / 2) != (b < n / 2)) ? 1 : 0;
            for (int l = 0; l < 9; ++l)
                for (int m = 0; m < 9; ++m) {
                    const double v = S.K[o][l][m] + beta * h * h * S.M[o][l][m];
                    for (int c = 0; c < 2; ++c) {
                        const int r = vidx(c, 2 * a + l % 3, 2 * b + l / 3), q = vidx(c, 2 * a + m % 3, 2 * b + m / 3);
                        if (r >= 0 && q >= 0) at(r, q) += v;
                    }
                }
            for (int q = 0; q < 4; ++q) {
                const int pr = pidx(a + q % 2, b + q / 2);
                for (int m = 0; m < 9; ++m) {
                    const int cx = vidx(0, 2 * a + m % 3, 2 * b + m / 3), cy = vidx(1, 2 * a + m % 3, 2 * b + m / 3);
                    if (cx >= 0) {
                        at(pr, cx) += h * S.Bx[o][q][m];
                        at(cx, pr) += h * S.Bx[o][q][m];
                    }
                    if (cy >= 0) {
                        at(pr, cy) += h * S.By[o][q][m];
                        at(cy, pr) += h * S.By[o][q][m];
                    }
                }
                double wq = 0.0;
                for (int r = 0; r < 4; ++r) wq += h * h * S.MP[o][q][r];
                at(pr, nb - 1) += wq;
                at(nb - 1, pr) += wq;
            }
        }
    for (int c = 0; c < 2; ++c)
        for (int Y = 1; Y < 2 * n; ++Y)
            for (int X = 1; X < 2 * n; ++X)
                if (!l_interior(X, Y, n)) {
                    const int r = c * nv + (Y - 1) * nm + (X - 1);
                    at(r, r) = 1.0;
                }
    for (int y = 0; y <= n; ++y)
        for (int x = 0; x <= n; ++x)
            if (2 * x > n && 2 * y > n) at(pidx(x, y), pidx(x, y)) = 1.0;
}

}  // namespace smg

extern "C" stokes_status stokes_lshape_vertex_rows(int levels, int kind, double* mbx, double* mby, double* w) {
    if (levels < 2 || levels > 13 || kind < 0 || kind >= kKinds || !mbx || !mby || !w) return STOKES_ERR_BAD_ARG;
    vertex_rows(squares_l(), 1 << levels, kind, mbx, mby, w);
    return STOKES_OK;
}

extern "C" stokes_status stokes_lshape_schur(int levels, double beta, double* s0, double* s1, double* s2) {
    if (levels < 2 || levels > 13 || !(beta >= 0.0) || !std::isfinite(beta) || !s0 || !s1 || !s2)
        return STOKES_ERR_BAD_ARG;
    const SquareMatrices& S = squares_l();
    const int n = 1 << levels, hn = n / 2;
    for (int kind = 0; kind < kKinds; ++kind) {
        double mbx[25], mby[25], w;
        vertex_rows(S, n, kind, mbx, mby, &w);
        // kinds 0 / 1: t = 0 .. hn - 2 of s0 / s1; kinds 3 / 4: their last entry t = hn - 1
        double* out = kind == 0 || kind == 3 ? s0 : kind == 1 || kind == 4 ? s1 : s2;
        const int t0 = kind >= 3 ? hn - 1 : 0, count = kind == 2 ? 1 : kind >= 3 ? 1 : hn - 1;
        for (int t = t0; t < t0 + count; ++t) {
            const bool side_x = kind == 0 || kind == 3, side_y = kind == 1 || kind == 4;
            const int i = side_y ? hn + 1 + t : hn, j = side_x ? hn + 1 + t : hn;
            double s = 0.0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx) {
                    const int X = 2 * i + dx, Y = 2 * j + dy;
                    if (!l_interior(X, Y, n)) continue;                 // Dirichlet or outside
                    const double bx = mbx[(dy + 2) * 5 + dx + 2], by = mby[(dy + 2) * 5 + dx + 2];
                    s += (bx * bx + by * by) / a_diag(S, X, Y, n, beta);
                }
            out[kind == 2 ? 0 : t] = s;
        }
    }
    return STOKES_OK;
}

// Level 0 of the L-shaped hierarchy is the square's level with N = 4 without the upper-right
// quadrant: the system of eq. gen:bil:mv over its 12 squares, Dirichlet velocity on the outer and
// re-entrant sides, bordered with w = M_P 1 (zero-mean pressure), inverted by Gauss-Jordan
// elimination with partial pivoting.  Unknowns: u_x at the interior nodes of the L in lattice order
// (Y outer), then u_y, then p at the vertices of the L in lattice order.
extern "C" stokes_status stokes_lshape_coarse_inverse(double beta, double* inv, int* nunk) {
    if (!inv || !nunk || !(beta >= 0.0) || !std::isfinite(beta)) return STOKES_ERR_BAD_ARG;
    const SquareMatrices& S = squares_l();
    const int n = 4, m2 = 2 * n + 1, m1 = n + 1;
    const double h = 1.0 / n;
    auto kept = [&](int a, int b) { return !(a >= n / 2 && b >= n / 2); };
    std::vector<int> vel(m2 * m2, -1), pre(m1 * m1, -1);
    int ni = 0;
    for (int Y = 0; Y < m2; ++Y)
        for (int X = 0; X < m2; ++X)
            if (l_interior(X, Y, n)) vel[Y * m2 + X] = ni++;
    std::vector<char> inl(m1 * m1, 0);
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a)
            if (kept(a, b))
                for (int q = 0; q < 4; ++q) inl[(b + q / 2) * m1 + a + q % 2] = 1;
    int np = 0;
    for (int v = 0; v < m1 * m1; ++v)
        if (inl[v]) pre[v] = 2 * ni + np++;
    const int nu = 2 * ni + np, nb = nu + 1;
    std::vector<double> M((size_t)nb * 2 * nb, 0.0);        // [A | I], row-major, width 2 nb
    auto at = [&](int r, int c) -> double& { return M[(size_t)r * 2 * nb + c]; };
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            if (!kept(a, b)) continue;
            const int o = ((a < n / 2) != (b < n / 2)) ? 1 : 0;
            int node[9];
            for (int l = 0; l < 9; ++l) node[l] = vel[(2 * b + l / 3) * m2 + 2 * a + l % 3];
            for (int l = 0; l < 9; ++l)
                for (int k = 0; k < 9; ++k)
                    if (node[l] >= 0 && node[k] >= 0) {
                        const double v = S.K[o][l][k] + beta * h * h * S.M[o][l][k];
                        at(node[l], node[k]) += v;
                        at(ni + node[l], ni + node[k]) += v;
                    }
            for (int q = 0; q < 4; ++q) {
                const int pr = pre[(b + q / 2) * m1 + a + q % 2];
                for (int k = 0; k < 9; ++k) {
                    if (node[k] < 0) continue;
                    at(pr, node[k]) += h * S.Bx[o][q][k];
                    at(node[k], pr) += h * S.Bx[o][q][k];
                    at(pr, ni + node[k]) += h * S.By[o][q][k];
                    at(ni + node[k], pr) += h * S.By[o][q][k];
                }
                for (int r = 0; r < 4; ++r) {
                    at(pr, nu) += h * h * S.MP[o][q][r];
                    at(nu, pr) += h * h * S.MP[o][q][r];
                }
            }
        }
    for (int i = 0; i < nb; ++i) at(i, nb + i) = 1.0;
    for (int c = 0; c < nb; ++c) {
        int piv = c;
        for (int r = c + 1; r < nb; ++r)
            if (std::fabs(at(r, c)) > std::fabs(at(piv, c))) piv = r;
        if (std::fabs(at(piv, c)) < 1e-300) return STOKES_ERR_BAD_ARG;
        if (piv != c)
            for (int k = 0; k < 2 * nb; ++k) std::swap(at(piv, k), at(c, k));
        const double d = at(c, c);
        for (int k = 0; k < 2 * nb; ++k) at(c, k) /= d;
        for (int r = 0; r < nb; ++r)
            if (r != c && at(r, c) != 0.0) {
                const double f = at(r, c);
                for (int k = 0; k < 2 * nb; ++k) at(r, k) -= f * at(c, k);
            }
    }
    for (int i = 0; i < nu; ++i)
        for (int k = 0; k < nu; ++k) inv[(size_t)i * nu + k] = at(i, nb + k);
    *nunk = nu;
    return STOKES_OK;
}
