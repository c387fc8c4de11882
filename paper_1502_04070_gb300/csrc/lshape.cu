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

#include "../../include/stokes_mg.h"
#include "common.cuh"
#include "elements.h"

using namespace smg;

namespace {

// Squares around vertex (i, j): SQ 0 = (i, j), 1 = (i-1, j), 2 = (i, j-1), 3 = (i-1, j-1); the vertex
// is corner SQ of square SQ.  Squares in the removed quadrant, per kind of re-entrant vertex:
//   kind 0, side x = 1/2 above the corner: SQ 0 and 2 (to the right);
//   kind 1, side y = 1/2 right of the corner: SQ 0 and 1 (above);
//   kind 2, the corner (1/2, 1/2): SQ 0.
// The stencil classes of these cells (the mid-line cells above / right of the centre, and the
// centre cell) give the orientation of every square.
constexpr unsigned kRemoved[3] = {0x5u, 0x3u, 0x1u};
constexpr int kClass[3] = {3, 5, 6};

// Velocity lattice node (X, Y) of the P2 lattice ([0, 2n]^2) strictly inside the L: off the outer
// boundary and off the closed removed quadrant (whose edges are the re-entrant sides).
bool l_interior(int X, int Y, int n) {
    if (X <= 0 || Y <= 0 || X >= 2 * n || Y >= 2 * n) return false;
    return !(X >= n && Y >= n);
}

// Diagonal of A = K + beta M at an interior lattice node: the sum over the squares that contain it
// (orientation 0 in the lower-left and upper-right quadrants, 1 in the other two, Sec. 5 mesh).
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

extern "C" stokes_status stokes_lshape_vertex_rows(int levels, int kind, double* mbx, double* mby, double* w) {
    if (levels < 2 || levels > 13 || kind < 0 || kind > 2 || !mbx || !mby || !w) return STOKES_ERR_BAD_ARG;
    vertex_rows(squares_l(), 1 << levels, kind, mbx, mby, w);
    return STOKES_OK;
}

extern "C" stokes_status stokes_lshape_schur(int levels, double beta, double* s0, double* s1, double* s2) {
    if (levels < 2 || levels > 13 || !(beta >= 0.0) || !std::isfinite(beta) || !s0 || !s1 || !s2)
        return STOKES_ERR_BAD_ARG;
    const SquareMatrices& S = squares_l();
    const int n = 1 << levels, hn = n / 2;
    double* out[3] = {s0, s1, s2};
    for (int kind = 0; kind < 3; ++kind) {
        double mbx[25], mby[25], w;
        vertex_rows(S, n, kind, mbx, mby, &w);
        const int count = kind == 2 ? 1 : hn - 1;
        for (int t = 0; t < count; ++t) {
            const int i = kind == 1 ? hn + 1 + t : hn, j = kind == 0 ? hn + 1 + t : hn;
            double s = 0.0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx) {
                    const int X = 2 * i + dx, Y = 2 * j + dy;
                    if (!l_interior(X, Y, n)) continue;                 // Dirichlet or outside
                    const double bx = mbx[(dy + 2) * 5 + dx + 2], by = mby[(dy + 2) * 5 + dx + 2];
                    s += (bx * bx + by * by) / a_diag(S, X, Y, n, beta);
                }
            out[kind][t] = s;
        }
    }
    return STOKES_OK;
}
