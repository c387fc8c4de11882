// common.cuh -- data structures and device helpers shared by the solver's kernels.
//
// Geometry (Sec. 6): level k of the unit square has N = 2^(k+1) squares per side; square (si, sj)
// covers [si/N, (si+1)/N] x [sj/N, (sj+1)/N] and is cut by one diagonal.  Refining the 8-triangle
// coarse mesh (the fan around the centre) keeps the diagonal direction of each quadrant:
//     orientation 0 ("/", from (0,0) to (1,1) of the square) in the SW and NE quadrants,
//     orientation 1 ("\", from (1,0) to (0,1))                in the SE and NW quadrants.
// A square carries 9 P2 nodes (local index m = 3*b + a at P2-lattice point (2si+a, 2sj+b)) and
// 4 P1 vertices (local q = 2*b' + a' at vertex (si+a', sj+b')).
//
// The operator of eq. gen:bil:mv is applied element-by-element per square ("matrix free"):
// a velocity row of A_k (= K + beta M_U, Sec. 2) is the sum, over the 1, 2 or 4 squares that
// contain the node, of one row of the square's 9x9 local matrix; likewise for B_k (4x9 per
// component) and B_k^T.  The local matrices are assembled on the host from exact P2/P1 element
// integrals and passed to kernels by value (constant bank).
//
// A thread "owns" cell (i, j), i, j in [0, N]: the vertex node V = (2i, 2j), the horizontal-edge
// node H = (2i+1, 2j), the vertical-edge node E = (2i, 2j+1), the centre node C = (2i+1, 2j+1)
// and the pressure vertex (i, j).  Nodes that fall outside the lattice do not exist.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace smg {

// Stencil classes of a cell by the orientations of its four squares (bit SQ of the pattern is the
// orientation of square SQ, numbered as in sq_local below: 0 = (i, j), 1 = (i-1, j), 2 = (i, j-1),
// 3 = (i-1, j-1)).  Classes 0 / 1: every cell off the two mid-lines (all four squares orientation
// 0 / 1).  On the mid-line x = 1/2 (i = N/2): class 2 below the centre, 3 above; on y = 1/2
// (j = N/2): class 4 left of the centre, 5 right; class 6 the centre cell.  Squares outside the
// domain get a pattern bit too: every lattice value they touch is a Dirichlet zero or outside the
// arrays (read as zero), so their terms vanish.
constexpr int kStencilClasses = 7;
__host__ __device__ constexpr unsigned stencil_pattern(int k) {
    return k == 0 ? 0x0u : k == 1 ? 0xFu : k == 2 ? 0x5u : k == 3 ? 0xAu : k == 4 ? 0x3u : k == 5 ? 0xCu : 0x6u;
}
__host__ __device__ constexpr int sq_orient(int k, int SQ) { return (int)((stencil_pattern(k) >> SQ) & 1u); }

template <typename T>
struct OpCoef {            // local square matrices of one level
    T A[2][9][9];          // K + beta h^2 Mhat        (h-independent stiffness, mass ~ h^2)
    T Bx[2][4][9];         // (d phi_m / dx, psi_q)    (~ h)
    T By[2][4][9];
    // The same operator as node stencils, per stencil class k: the rows of the four owned velocity
    // nodes s (V, H, E, C) over the 5 x 5 lattice window of the cell (offsets dx, dy in -2..2 from
    // (2i, 2j)), their B^T rows over the 3 x 3 vertex window, and the B row of the owned vertex.
    // Built by fill_merged().
    T MA[kStencilClasses][4][25];    // [k][s][(dy+2)*5 + dx+2]
    T MBTx[kStencilClasses][4][9];   // [k][s][(dj+1)*3 + di+1]
    T MBTy[kStencilClasses][4][9];
    T MBx[kStencilClasses][25];      // [k][(dy+2)*5 + dx+2]
    T MBy[kStencilClasses][25];
    T MIdg[kStencilClasses][4];      // 1 / diag A of the four owned nodes, [k][s]
};

template <typename T>
struct MassCoef {          // mass matrices of one level (load vectors, adjoint)
    T M[2][9][9];
    T MP[2][4][4];
};

// triangle membership of local P2 nodes, per orientation (bit m set if node m lies in the triangle)
//  o = 0: T0 = {(0,0),(2,0),(2,2)} -> nodes {0,1,2,4,5,8};  T1 = {(0,0),(2,2),(0,2)} -> {0,3,4,6,7,8}
//  o = 1: T0 = {(0,0),(2,0),(0,2)} -> nodes {0,1,2,3,4,6};  T1 = {(2,0),(2,2),(0,2)} -> {2,4,5,6,7,8}
__host__ __device__ constexpr unsigned tri_mask(int o, int t) {
    return o == 0 ? (t == 0 ? 0x137u : 0x1D9u) : (t == 0 ? 0x05Fu : 0x1F4u);
}
__host__ __device__ constexpr bool couple(int o, int l, int m) {
    return (((tri_mask(o, 0) >> l) & 1u) && ((tri_mask(o, 0) >> m) & 1u)) ||
           (((tri_mask(o, 1) >> l) & 1u) && ((tri_mask(o, 1) >> m) & 1u));
}
__host__ __device__ constexpr int corner_node(int q) { return q == 0 ? 0 : q == 1 ? 2 : q == 2 ? 6 : 8; }

// Squares around cell (i, j): SQ 0 = (i, j), 1 = (i-1, j), 2 = (i, j-1), 3 = (i-1, j-1); the
// cell's vertex is corner SQ of square SQ.  Owned node s (0 V, 1 H, 2 E, 3 C) sits at local node
// sq_local(SQ, s) of square SQ, or -1 if the square does not contain it.
__host__ __device__ constexpr int sq_local(int SQ, int s) {
    // node offset from the cell origin (2i, 2j): (s & 1, s >> 1); square origin: (-2 (SQ & 1), -2 (SQ >> 1))
    return ((s & 1) + 2 * (SQ & 1) > 2 || (s >> 1) + 2 * (SQ >> 1) > 2)
               ? -1
               : 3 * ((s >> 1) + 2 * (SQ >> 1)) + (s & 1) + 2 * (SQ & 1);
}
// lattice offset (from (2i, 2j)) of local node m of square SQ, as a 5 x 5 window index
__host__ __device__ constexpr int sq_win(int SQ, int m) { return (m / 3 - 2 * (SQ >> 1) + 2) * 5 + (m % 3 - 2 * (SQ & 1) + 2); }
// vertex offset (from (i, j)) of corner q of square SQ, as a 3 x 3 window index
__host__ __device__ constexpr int sq_vwin(int SQ, int q) { return (q / 2 - (SQ >> 1) + 1) * 3 + (q % 2 - (SQ & 1) + 1); }

// structural nonzeros of the merged stencils of class k (compile-time)
__host__ __device__ constexpr bool nz_MA(int k, int s, int w) {
    for (int SQ = 0; SQ < 4; ++SQ) {
        const int L = sq_local(SQ, s);
        if (L < 0) continue;
        for (int m = 0; m < 9; ++m)
            if (sq_win(SQ, m) == w && couple(sq_orient(k, SQ), L, m)) return true;
    }
    return false;
}
__host__ __device__ constexpr bool nz_MBT(int k, int s, int v) {
    for (int SQ = 0; SQ < 4; ++SQ) {
        const int L = sq_local(SQ, s);
        if (L < 0) continue;
        for (int q = 0; q < 4; ++q)
            if (sq_vwin(SQ, q) == v && couple(sq_orient(k, SQ), corner_node(q), L)) return true;
    }
    return false;
}
__host__ __device__ constexpr bool nz_MB(int k, int w) {
    for (int SQ = 0; SQ < 4; ++SQ)
        for (int m = 0; m < 9; ++m)
            if (sq_win(SQ, m) == w && couple(sq_orient(k, SQ), corner_node(SQ), m)) return true;
    return false;
}

// host: merged stencils from the square-local matrices (sums over the squares that share a node)
template <typename T>
inline void fill_merged(OpCoef<T>& c) {
    for (int k = 0; k < kStencilClasses; ++k) {
        for (int s = 0; s < 4; ++s) {
            double ma[25] = {}, bx[9] = {}, by[9] = {};
            for (int SQ = 0; SQ < 4; ++SQ) {
                const int L = sq_local(SQ, s), o = sq_orient(k, SQ);
                if (L < 0) continue;
                for (int m = 0; m < 9; ++m)
                    if (couple(o, L, m)) ma[sq_win(SQ, m)] += (double)c.A[o][L][m];
                for (int q = 0; q < 4; ++q)
                    if (couple(o, corner_node(q), L)) {
                        bx[sq_vwin(SQ, q)] += (double)c.Bx[o][q][L];
                        by[sq_vwin(SQ, q)] += (double)c.By[o][q][L];
                    }
            }
            for (int w = 0; w < 25; ++w) c.MA[k][s][w] = (T)ma[w];
            c.MIdg[k][s] = (T)(1.0 / ma[((s >> 1) + 2) * 5 + (s & 1) + 2]);
            for (int v = 0; v < 9; ++v) {
                c.MBTx[k][s][v] = (T)bx[v];
                c.MBTy[k][s][v] = (T)by[v];
            }
        }
        double mx[25] = {}, my[25] = {};
        for (int SQ = 0; SQ < 4; ++SQ) {
            const int o = sq_orient(k, SQ);
            for (int m = 0; m < 9; ++m)
                if (couple(o, corner_node(SQ), m)) {
                    mx[sq_win(SQ, m)] += (double)c.Bx[o][SQ][m];
                    my[sq_win(SQ, m)] += (double)c.By[o][SQ][m];
                }
        }
        for (int w = 0; w < 25; ++w) {
            c.MBx[k][w] = (T)mx[w];
            c.MBy[k][w] = (T)my[w];
        }
    }
}

__host__ __device__ __forceinline__ int orient(int si, int sj, int n) {
    const int h = n >> 1;
    return (si < h) != (sj < h);
}

// number of triangles at vertex (i, j) of a level with N = n (0 outside the level)
__device__ __forceinline__ int vertex_triangles(int i, int j, int n) {
    int cnt = 0;
#pragma unroll
    for (int SQ = 0; SQ < 4; ++SQ) {
        const int si = i - (SQ & 1), sj = j - (SQ >> 1);
        if (si < 0 || sj < 0 || si >= n || sj >= n) continue;
        const int o = orient(si, sj, n), node = corner_node(SQ);
        cnt += ((tri_mask(o, 0) >> node) & 1u) + ((tri_mask(o, 1) >> node) & 1u);
    }
    return cnt;
}

// w_i = int psi_i = (number of triangles at vertex i) h^2 / 6: the pressure-mean weight (M_P 1)_i
__device__ __forceinline__ double vertex_weight(int i, int j, int n) {
    const double h = 1.0 / n;
    return vertex_triangles(i, j, n) * h * h / 6.0;
}

// stencil class (see stencil_pattern) of cell (i, j) of a level with N = n
__host__ __device__ __forceinline__ int stencil_class(int i, int j, int n) {
    const int h = n >> 1;
    if (i != h && j != h) return orient(i, j, n);
    if (i == h && j == h) return 6;
    if (i == h) return j < h ? 2 : 3;
    return i < h ? 4 : 5;
}

// row L of A (orientation O) times the 9 square values; zero couplings dropped at compile time
template <int O, int L, int M, typename T>
__device__ __forceinline__ void a_term(const T (&A)[2][9][9], const T (&v)[9], T& s) {
    if constexpr (couple(O, L, M)) s = fma(A[O][L][M], v[M], s);
}
template <int O, int L, typename T, int... M>
__device__ __forceinline__ T arow_i(const T (&A)[2][9][9], const T (&v)[9], std::integer_sequence<int, M...>) {
    T s = T(0);
    (a_term<O, L, M>(A, v, s), ...);
    return s;
}
template <int O, int L, typename T>
__device__ __forceinline__ T arow(const T (&A)[2][9][9], const T (&v)[9]) {
    return arow_i<O, L>(A, v, std::make_integer_sequence<int, 9>{});
}
// (B^T p) restricted to row L: sum_q B[q][L] p[q]
template <int O, int L, int Q, typename T>
__device__ __forceinline__ void bt_term(const T (&B)[2][4][9], const T (&p)[4], T& s) {
    if constexpr (couple(O, corner_node(Q), L)) s = fma(B[O][Q][L], p[Q], s);
}
template <int O, int L, typename T>
__device__ __forceinline__ T btrow(const T (&B)[2][4][9], const T (&p)[4]) {
    T s = T(0);
    bt_term<O, L, 0>(B, p, s);
    bt_term<O, L, 1>(B, p, s);
    bt_term<O, L, 2>(B, p, s);
    bt_term<O, L, 3>(B, p, s);
    return s;
}
// (B u) restricted to pressure row Q
template <int O, int Q, int M, typename T>
__device__ __forceinline__ void b_term(const T (&B)[2][4][9], const T (&v)[9], T& s) {
    if constexpr (couple(O, corner_node(Q), M)) s = fma(B[O][Q][M], v[M], s);
}
template <int O, int Q, typename T, int... M>
__device__ __forceinline__ T brow_i(const T (&B)[2][4][9], const T (&v)[9], std::integer_sequence<int, M...>) {
    T s = T(0);
    (b_term<O, Q, M>(B, v, s), ...);
    return s;
}
template <int O, int Q, typename T>
__device__ __forceinline__ T brow(const T (&B)[2][4][9], const T (&v)[9]) {
    return brow_i<O, Q>(B, v, std::make_integer_sequence<int, 9>{});
}

// Is P2-lattice point (X, Y) an interior velocity node of a level with N = n?
__device__ __forceinline__ bool interior2(int X, int Y, int n) {
    return X > 0 && Y > 0 && X < 2 * n && Y < 2 * n;
}

// Which owned nodes of cell (i, j) exist / are unknowns.
struct CellNodes {
    bool v, h, e, c;   // unknown velocity nodes
    bool hx, ex, cx;   // node exists in the lattice (may be a boundary node)
};
__device__ __forceinline__ CellNodes cell_nodes(int i, int j, int n) {
    CellNodes c;
    c.hx = i < n;
    c.ex = j < n;
    c.cx = i < n && j < n;
    c.v = i > 0 && j > 0 && i < n && j < n;
    c.h = c.hx && j > 0 && j < n;
    c.e = c.ex && i > 0 && i < n;
    c.c = c.cx;
    return c;
}

// The L-shaped domain (the unit square without its upper-right quadrant [1/2, 1]^2) on the square's
// lattice: velocity nodes in the closed removed quadrant (lattice X >= N and Y >= N, its edges being
// the re-entrant sides) are Dirichlet nodes, and vertices strictly inside it (i > N/2, j > N/2) are
// not pressure unknowns.  Every other node keeps the square's rows: all triangles around a velocity
// node strictly inside the L lie in the L.
enum : int { kDomSquare = 0, kDomL = 1 };
__host__ __device__ __forceinline__ bool l_masked_node(int X, int Y, int n) { return X >= n && Y >= n; }
__host__ __device__ __forceinline__ bool l_masked_vertex(int i, int j, int n) { return 2 * i > n && 2 * j > n; }
__device__ __forceinline__ CellNodes cell_nodes_dom(int i, int j, int n, int dom) {
    CellNodes c = cell_nodes(i, j, n);
    if (dom == kDomL) {
        c.v = c.v && !l_masked_node(2 * i, 2 * j, n);
        c.h = c.h && !l_masked_node(2 * i + 1, 2 * j, n);
        c.e = c.e && !l_masked_node(2 * i, 2 * j + 1, n);
        c.c = c.c && !l_masked_node(2 * i + 1, 2 * j + 1, n);
    }
    return c;
}
// number of triangles at vertex (i, j) on the square or the L (squares of the removed quadrant do
// not count)
__device__ __forceinline__ int vertex_triangles_dom(int i, int j, int n, int dom) {
    if (dom != kDomL) return vertex_triangles(i, j, n);
    int cnt = 0;
#pragma unroll
    for (int SQ = 0; SQ < 4; ++SQ) {
        const int si = i - (SQ & 1), sj = j - (SQ >> 1);
        if (si < 0 || sj < 0 || si >= n || sj >= n || (2 * si >= n && 2 * sj >= n)) continue;
        const int o = orient(si, sj, n), node = corner_node(SQ);
        cnt += ((tri_mask(o, 0) >> node) & 1u) + ((tri_mask(o, 1) >> node) & 1u);
    }
    return cnt;
}
// w_i = int_Omega psi_i for the square or the L
__device__ __forceinline__ double vertex_weight_dom(int i, int j, int n, int dom) {
    const double h = 1.0 / n;
    return vertex_triangles_dom(i, j, n, dom) * h * h / 6.0;
}

// Planar float32 layout of the large float32 levels (the velocity arrays of the refinement's inner
// cycles, staged by the tensor-memory-access engine, which needs 16-byte row pitches):
//   velocity: (u_x, u_y) pairs side by side, in two planes by the parity of the lattice column X;
//             plane a holds the points X = 2 q + a, row Y at pair q; pl_rows(n) = 2N + 2 rows per
//             plane (row 2N + 1 is padding) of pl_pitch(n) = N + 2 pairs (q = N + 1, and q = N of
//             plane 1, are padding), so every row starts on a 16-byte boundary;
//   vertex arrays: rows of pl_vpitch(n) = N + 1 rounded up to 4 floats.
// Padding and the Dirichlet boundary nodes of every velocity array hold zero (the arrays are zeroed
// when allocated, and kernels write the boundary nodes as zero and never write the padding), so a
// tile of either plane, or of the four node-type planes, is one box copy with no masking.
__host__ __device__ __forceinline__ int pl_pitch(int n) { return (n + 2) & ~1; }
__host__ __device__ __forceinline__ int pl_rows(int n) { return 2 * n + 2; }
__host__ __device__ __forceinline__ int pl_vpitch(int n) { return (n + 4) & ~3; }
__host__ __device__ __forceinline__ size_t pl_ucount(int n) { return (size_t)4 * pl_rows(n) * pl_pitch(n); }   // floats
__host__ __device__ __forceinline__ size_t pl_pcount(int n) { return (size_t)(n + 1) * pl_vpitch(n); }
// float index of u_x at lattice point (X, Y); u_y follows it
__host__ __device__ __forceinline__ int pl_u(int n, int X, int Y) {
    return (((X & 1) * pl_rows(n) + Y) * pl_pitch(n) + (X >> 1)) * 2;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Block-wide sum of one double per thread; returns the total in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        s = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

}  // namespace smg
