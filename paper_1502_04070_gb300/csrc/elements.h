// elements.h -- host-side construction of the local matrices used by the kernels.
#pragma once

namespace smg {

// Local matrices of one square with leg h = 1, for both orientations o (see common.cuh).
// On a level with leg h:  K scales as h^0, M as h^2, Bx/By as h, MP as h^2.
struct SquareMatrices {
    double K[2][9][9];
    double M[2][9][9];
    double Bx[2][4][9];
    double By[2][4][9];
    double MP[2][4][4];
};

// Canonical P2 embedding weights: value of coarse local basis function L (0..8) of a coarse
// square of orientation o at its fine lattice point (fa, fb), fa, fb in [0, 4].
struct TransferWeights {
    double P2[2][9][5][5];
};

SquareMatrices square_matrices();
TransferWeights transfer_weights();

// Inverse (first 27 x 27 block) of the level-0 system bordered with the zero-mean constraint.
bool coarse_inverse(const SquareMatrices& S, double beta, double inv[27 * 27]);

// Size nb and row-major entries (caller array of nb * nb) of the system of a level with N = n
// bordered with the zero-mean pressure condition (unknown order as in coarse_inverse).
int bordered_size(int n);
void bordered_system(const SquareMatrices& S, int n, double beta, double* M);
// Level 0 of the L-shaped hierarchy (the square's level with N = 4 without its upper-right quadrant)
// in the same order and size (n = 4), with identity rows at the square's unknowns outside the L.
void lshape_bordered_system(double beta, double* M);

}  // namespace smg
