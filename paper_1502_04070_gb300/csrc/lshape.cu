// lshape.cu -- host tables for the L-shaped domain (the unit square without [1/2, 1]^2).
//
// Sec. 1: the convergence theory needs a convex domain, the method does not.  On the L the square's
// lattice and node stencils carry over unchanged at every velocity node strictly inside the L (all
// of its triangles lie in the L); the nodes on the re-entrant sides x = 1/2 (y >= 1/2) and
// y = 1/2 (x >= 1/2) join the Dirichlet set.  The pressure vertices on those sides stay unknowns,
// and their B rows and pressure-mass weights sum over the squares around the vertex that lie in
// the L only: this file computes those rows from the same square matrices as the square's tables.
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

}  // namespace

extern "C" stokes_status stokes_lshape_vertex_rows(int levels, int kind, double* mbx, double* mby, double* w) {
    if (levels < 2 || levels > 13 || kind < 0 || kind > 2 || !mbx || !mby || !w) return STOKES_ERR_BAD_ARG;
    const int n = 1 << levels;
    const double h = 1.0 / n;
    static const SquareMatrices S = square_matrices();
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
    return STOKES_OK;
}
