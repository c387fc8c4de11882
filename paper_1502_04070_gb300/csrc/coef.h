// coef.h -- host construction of a level's operator and mass coefficients (used by every entry point
// that launches operator kernels, so that all of them apply the same matrices).
#pragma once
#include "common.cuh"
#include "elements.h"

namespace smg {

// Local matrices of the unit square (exact P2/P1 element integrals, elements.cpp), built once per
// process.
inline const SquareMatrices& square_tables() {
    static const SquareMatrices S = square_matrices();
    return S;
}

// The operator of eq. gen:bil:mv on a level with N = n squares per side (leg h = 1/n): the square's
// A = K + beta h^2 M (K is scale-free in 2D, M scales with h^2), Bx, By scaled with h, and the merged
// node stencils of the seven stencil classes.
template <typename T>
OpCoef<T> make_coef(int n, double beta) {
    const SquareMatrices& S = square_tables();
    const double h = 1.0 / n;
    OpCoef<T> c;
    for (int o = 0; o < 2; ++o) {
        for (int l = 0; l < 9; ++l)
            for (int m = 0; m < 9; ++m) c.A[o][l][m] = (T)(S.K[o][l][m] + beta * h * h * S.M[o][l][m]);
        for (int q = 0; q < 4; ++q)
            for (int m = 0; m < 9; ++m) {
                c.Bx[o][q][m] = (T)(h * S.Bx[o][q][m]);
                c.By[o][q][m] = (T)(h * S.By[o][q][m]);
            }
    }
    fill_merged(c);
    return c;
}

// Velocity and pressure mass matrices of one square on a level with N = n (load vectors, adjoint).
template <typename T>
MassCoef<T> make_mass(int n) {
    const SquareMatrices& S = square_tables();
    const double h = 1.0 / n;
    MassCoef<T> m;
    for (int o = 0; o < 2; ++o) {
        for (int l = 0; l < 9; ++l)
            for (int k = 0; k < 9; ++k) m.M[o][l][k] = (T)(h * h * S.M[o][l][k]);
        for (int q = 0; q < 4; ++q)
            for (int r = 0; r < 4; ++r) m.MP[o][q][r] = (T)(h * h * S.MP[o][q][r]);
    }
    return m;
}

}  // namespace smg
