// elements.cpp -- local P2/P1 square matrices, transfer weights and the level-0 system (host).
//
// Element integrals (Sec. 2): a(u, v) = (grad u, grad v) + beta (u, v), b(u, q) = (div u, q).
// Basis functions in barycentric coordinates (lambda_0, lambda_1, lambda_2) of a triangle:
//   P2 vertex i: lambda_i (2 lambda_i - 1),  P2 edge (i, j): 4 lambda_i lambda_j,  P1 vertex i: lambda_i,
// and every integral is exact via  int_T lambda^a = 2|T| a0! a1! a2! / (a0 + a1 + a2 + 2)!.
// A square of the structured mesh holds two triangles; its 9x9 / 4x9 local matrices are the sums
// of the two element matrices (see common.cuh for the local numbering and orientations).
#include "elements.h"

#include <array>
#include <cmath>
#include <cstring>
#include <vector>

namespace smg {
namespace {

struct Mono {
    int e[3];
    double c;
};
using Poly = std::vector<Mono>;

Poly mul(const Poly& a, const Poly& b) {
    Poly out;
    for (const Mono& x : a)
        for (const Mono& y : b) {
            Mono z{{x.e[0] + y.e[0], x.e[1] + y.e[1], x.e[2] + y.e[2]}, x.c * y.c};
            bool merged = false;
            for (Mono& w : out)
                if (w.e[0] == z.e[0] && w.e[1] == z.e[1] && w.e[2] == z.e[2]) {
                    w.c += z.c;
                    merged = true;
                    break;
                }
            if (!merged) out.push_back(z);
        }
    return out;
}

Poly deriv(const Poly& a, int i) {
    Poly out;
    for (const Mono& x : a)
        if (x.e[i] > 0) {
            Mono z = x;
            z.c *= x.e[i];
            z.e[i] -= 1;
            out.push_back(z);
        }
    return out;
}

double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }

// int_T p / (2|T|)
double integ(const Poly& p) {
    double s = 0.0;
    for (const Mono& x : p) s += x.c * fact(x.e[0]) * fact(x.e[1]) * fact(x.e[2]) / fact(x.e[0] + x.e[1] + x.e[2] + 2);
    return s;
}

Poly lam(int i) {
    Mono m{{0, 0, 0}, 1.0};
    m.e[i] = 1;
    return Poly{m};
}

// local P2 order: v0, v1, v2, m12, m02, m01
std::array<Poly, 6> p2() {
    std::array<Poly, 6> b;
    for (int i = 0; i < 3; ++i) {
        Poly t = lam(i);
        t[0].c = 2.0;
        Poly lin = {Mono{{0, 0, 0}, -1.0}};
        lin.push_back(t[0]);
        b[i] = mul(lam(i), lin);
    }
    const int pr[3][2] = {{1, 2}, {0, 2}, {0, 1}};
    for (int k = 0; k < 3; ++k) {
        Poly t = mul(lam(pr[k][0]), lam(pr[k][1]));
        for (Mono& m : t) m.c *= 4.0;
        b[3 + k] = t;
    }
    return b;
}

double evalp(const Poly& p, const double l[3]) {
    double s = 0.0;
    for (const Mono& m : p) s += m.c * std::pow(l[0], m.e[0]) * std::pow(l[1], m.e[1]) * std::pow(l[2], m.e[2]);
    return s;
}

struct Elem {
    double K[6][6], M[6][6], Bx[3][6], By[3][6], MP[3][3];
};

// exact element matrices of the triangle with counter-clockwise vertices x[3], y[3]
Elem element(const double x[3], const double y[3]) {
    Elem E;
    const double twoA = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    double g[3][2];
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        g[i][0] = (y[j] - y[k]) / twoA;
        g[i][1] = (x[k] - x[j]) / twoA;
    }
    auto B = p2();
    Poly D[6][3];
    for (int a = 0; a < 6; ++a)
        for (int i = 0; i < 3; ++i) D[a][i] = deriv(B[a], i);
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            double k = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double G = g[i][0] * g[j][0] + g[i][1] * g[j][1];
                    if (G != 0.0) k += G * integ(mul(D[a][i], D[b][j]));
                }
            E.K[a][b] = twoA * k;
            E.M[a][b] = twoA * integ(mul(B[a], B[b]));
        }
    for (int q = 0; q < 3; ++q) {
        for (int b = 0; b < 6; ++b) {
            double bx = 0.0, by = 0.0;
            for (int i = 0; i < 3; ++i) {
                const double v = integ(mul(lam(q), D[b][i]));
                bx += g[i][0] * v;
                by += g[i][1] * v;
            }
            E.Bx[q][b] = twoA * bx;
            E.By[q][b] = twoA * by;
        }
        for (int r = 0; r < 3; ++r) E.MP[q][r] = twoA * integ(mul(lam(q), lam(r)));
    }
    return E;
}

// Triangles of a square in local half-leg units (corners at 0 and 2), counter-clockwise.
//  o = 0 ("/"): {(0,0),(2,0),(2,2)}, {(0,0),(2,2),(0,2)}
//  o = 1 ("\"): {(0,0),(2,0),(0,2)}, {(2,0),(2,2),(0,2)}
const int kTri[2][2][3][2] = {
    {{{0, 0}, {2, 0}, {2, 2}}, {{0, 0}, {2, 2}, {0, 2}}},
    {{{0, 0}, {2, 0}, {0, 2}}, {{2, 0}, {2, 2}, {0, 2}}},
};

int node_of(int a, int b) { return 3 * b + a; }
int corner_of(int a, int b) { return (b / 2) * 2 + a / 2; }

}  // namespace

SquareMatrices square_matrices() {
    SquareMatrices S;
    std::memset(&S, 0, sizeof(S));
    for (int o = 0; o < 2; ++o)
        for (int t = 0; t < 2; ++t) {
            double x[3], y[3];
            int loc[6], cor[3];
            for (int v = 0; v < 3; ++v) {
                x[v] = 0.5 * kTri[o][t][v][0];          // leg h = 1
                y[v] = 0.5 * kTri[o][t][v][1];
                loc[v] = node_of(kTri[o][t][v][0], kTri[o][t][v][1]);
                cor[v] = corner_of(kTri[o][t][v][0], kTri[o][t][v][1]);
            }
            const int pr[3][2] = {{1, 2}, {0, 2}, {0, 1}};
            for (int k = 0; k < 3; ++k) {
                const int a = (kTri[o][t][pr[k][0]][0] + kTri[o][t][pr[k][1]][0]) / 2;
                const int b = (kTri[o][t][pr[k][0]][1] + kTri[o][t][pr[k][1]][1]) / 2;
                loc[3 + k] = node_of(a, b);
            }
            Elem E = element(x, y);
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) {
                    S.K[o][loc[a]][loc[b]] += E.K[a][b];
                    S.M[o][loc[a]][loc[b]] += E.M[a][b];
                }
            for (int q = 0; q < 3; ++q) {
                for (int b = 0; b < 6; ++b) {
                    S.Bx[o][cor[q]][loc[b]] += E.Bx[q][b];
                    S.By[o][cor[q]][loc[b]] += E.By[q][b];
                }
                for (int r = 0; r < 3; ++r) S.MP[o][cor[q]][cor[r]] += E.MP[q][r];
            }
        }
    return S;
}

TransferWeights transfer_weights() {
    // Canonical embedding (Sec. 3): value of coarse basis function L of a coarse square at fine
    // lattice point (fa, fb) in [0, 4]^2 of that square (coarse corners at 0 and 4).
    TransferWeights W;
    std::memset(&W, 0, sizeof(W));
    auto B = p2();
    for (int o = 0; o < 2; ++o)
        for (int fb = 0; fb <= 4; ++fb)
            for (int fa = 0; fa <= 4; ++fa) {
                const double px = fa / 4.0, py = fb / 4.0;
                for (int t = 0; t < 2; ++t) {
                    double x[3], y[3];
                    for (int v = 0; v < 3; ++v) {
                        x[v] = 0.5 * kTri[o][t][v][0];
                        y[v] = 0.5 * kTri[o][t][v][1];
                    }
                    const double twoA = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
                    double l[3];
                    for (int i = 0; i < 3; ++i) {
                        const int j = (i + 1) % 3, k = (i + 2) % 3;
                        l[i] = ((x[j] - px) * (y[k] - py) - (x[k] - px) * (y[j] - py)) / twoA;
                    }
                    if (l[0] < -1e-12 || l[1] < -1e-12 || l[2] < -1e-12) continue;   // outside
                    int loc[6];
                    for (int v = 0; v < 3; ++v) loc[v] = node_of(kTri[o][t][v][0], kTri[o][t][v][1]);
                    const int pr[3][2] = {{1, 2}, {0, 2}, {0, 1}};
                    for (int k = 0; k < 3; ++k)
                        loc[3 + k] = node_of((kTri[o][t][pr[k][0]][0] + kTri[o][t][pr[k][1]][0]) / 2,
                                             (kTri[o][t][pr[k][0]][1] + kTri[o][t][pr[k][1]][1]) / 2);
                    for (int a = 0; a < 6; ++a) W.P2[o][loc[a]][fb][fa] = evalp(B[a], l);
                }
            }
    return W;
}

// Level 0 (N = 2): assemble the 27 x 27 system of eq. gen:bil:mv from the square matrices, border
// it with w = M_P 1 (zero-mean pressure) and invert the 28 x 28 matrix by Gauss-Jordan elimination
// with partial pivoting.  Unknown order: u_x at interior lattice points (X, Y) in [1, 3]^2 row-major,
// then u_y, then p at the 3 x 3 vertices row-major.  Returns false if singular.
bool coarse_inverse(const SquareMatrices& S, double beta, double inv[27 * 27]) {
    const int n = 2, nb = 28;
    double Abig[28][28] = {};
    auto vidx = [&](int c, int X, int Y) -> int {
        if (X <= 0 || Y <= 0 || X >= 2 * n || Y >= 2 * n) return -1;
        return c * 9 + (Y - 1) * 3 + (X - 1);
    };
    auto pidx = [&](int x, int y) { return 18 + y * 3 + x; };
    double w[9] = {};
    const double h = 1.0 / n;
    for (int sj = 0; sj < n; ++sj)
        for (int si = 0; si < n; ++si) {
            const int o = ((si < n / 2) != (sj < n / 2)) ? 1 : 0;
            for (int l = 0; l < 9; ++l)
                for (int m = 0; m < 9; ++m) {
                    const double a = S.K[o][l][m] + beta * h * h * S.M[o][l][m];
                    for (int c = 0; c < 2; ++c) {
                        const int r = vidx(c, 2 * si + l % 3, 2 * sj + l / 3);
                        const int q = vidx(c, 2 * si + m % 3, 2 * sj + m / 3);
                        if (r >= 0 && q >= 0) Abig[r][q] += a;
                    }
                }
            for (int q = 0; q < 4; ++q) {
                const int pr = pidx(si + q % 2, sj + q / 2);
                for (int m = 0; m < 9; ++m) {
                    const int cx = vidx(0, 2 * si + m % 3, 2 * sj + m / 3);
                    const int cy = vidx(1, 2 * si + m % 3, 2 * sj + m / 3);
                    if (cx >= 0) {
                        Abig[pr][cx] += h * S.Bx[o][q][m];
                        Abig[cx][pr] += h * S.Bx[o][q][m];
                    }
                    if (cy >= 0) {
                        Abig[pr][cy] += h * S.By[o][q][m];
                        Abig[cy][pr] += h * S.By[o][q][m];
                    }
                }
                for (int r = 0; r < 4; ++r) w[pr - 18] += h * h * S.MP[o][q][r];
            }
        }
    for (int i = 0; i < 9; ++i) {
        Abig[18 + i][27] = w[i];
        Abig[27][18 + i] = w[i];
    }
    // Gauss-Jordan on [Abig | I]
    double aug[28][56];
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < 2 * nb; ++j) aug[i][j] = j < nb ? Abig[i][j] : (j - nb == i ? 1.0 : 0.0);
    for (int c = 0; c < nb; ++c) {
        int piv = c;
        for (int r = c + 1; r < nb; ++r)
            if (std::fabs(aug[r][c]) > std::fabs(aug[piv][c])) piv = r;
        if (std::fabs(aug[piv][c]) < 1e-300) return false;
        if (piv != c)
            for (int j = 0; j < 2 * nb; ++j) std::swap(aug[piv][j], aug[c][j]);
        const double d = aug[c][c];
        for (int j = 0; j < 2 * nb; ++j) aug[c][j] /= d;
        for (int r = 0; r < nb; ++r)
            if (r != c && aug[r][c] != 0.0) {
                const double f = aug[r][c];
                for (int j = 0; j < 2 * nb; ++j) aug[r][j] -= f * aug[c][j];
            }
    }
    for (int i = 0; i < 27; ++i)
        for (int j = 0; j < 27; ++j) inv[i * 27 + j] = aug[i][nb + j];
    return true;
}

int bordered_size(int n) { return 2 * (2 * n - 1) * (2 * n - 1) + (n + 1) * (n + 1) + 1; }

// The matrix of eq. gen:bil:mv on a level with N = n, assembled square by square from the local
// matrices, bordered with w = M_P 1 (the zero-mean pressure condition): row-major nb x nb,
// nb = bordered_size(n).  Unknown order as in coarse_inverse: u_x at the interior lattice points
// (X, Y), 1 <= X, Y <= 2n - 1, Y outer; then u_y; then p at the vertices (x, y), y outer; then the
// border's multiplier.
void bordered_system(const SquareMatrices& S, int n, double beta, double* M) {
    const int nm = 2 * n - 1, nv = nm * nm, nb = bordered_size(n);
    std::memset(M, 0, sizeof(double) * (size_t)nb * nb);
    auto at = [&](int r, int c) -> double& { return M[(size_t)r * nb + c]; };
    auto vidx = [&](int c, int X, int Y) -> int {
        if (X <= 0 || Y <= 0 || X >= 2 * n || Y >= 2 * n) return -1;
        return c * nv + (Y - 1) * nm + (X - 1);
    };
    auto pidx = [&](int x, int y) { return 2 * nv + y * (n + 1) + x; };
    const double h = 1.0 / n;
    for (int sj = 0; sj < n; ++sj)
        for (int si = 0; si < n; ++si) {
            const int o = ((si < n / 2) != (sj < n / 2)) ? 1 : 0;
            for (int l = 0; l < 9; ++l)
                for (int m = 0; m < 9; ++m) {
                    const double a = S.K[o][l][m] + beta * h * h * S.M[o][l][m];
                    if (a == 0.0) continue;
                    for (int c = 0; c < 2; ++c) {
                        const int r = vidx(c, 2 * si + l % 3, 2 * sj + l / 3);
                        const int q = vidx(c, 2 * si + m % 3, 2 * sj + m / 3);
                        if (r >= 0 && q >= 0) at(r, q) += a;
                    }
                }
            for (int q = 0; q < 4; ++q) {
                const int pr = pidx(si + q % 2, sj + q / 2);
                for (int m = 0; m < 9; ++m) {
                    const int cx = vidx(0, 2 * si + m % 3, 2 * sj + m / 3);
                    const int cy = vidx(1, 2 * si + m % 3, 2 * sj + m / 3);
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
}

}  // namespace smg
