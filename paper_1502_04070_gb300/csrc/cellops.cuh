// cellops.cuh -- per-cell gather of operator rows (see common.cuh for the cell / square layout).
//
// A "view" maps P2-lattice coordinates (X, Y) (or vertex coordinates for pressure) to values; the
// same row code reads global memory through the read-only path or a shared-memory tile.
#pragma once
#include <utility>

#include "common.cuh"

namespace smg {

constexpr int BX = 32, BY = 8, NT = BX * BY;

int cells_blocks(int n);
inline dim3 cells_grid(int n) { return dim3((n + 1 + BX - 1) / BX, (n + 1 + BY - 1) / BY); }

// ------------------------------------------------------------------------------------------
// rows of the square at position SQ relative to the cell: SQ 0 = (i, j), 1 = (i-1, j),
// 2 = (i, j-1), 3 = (i-1, j-1).  The cell's vertex is corner Q = SQ of that square.
__host__ __device__ constexpr int sq_nrows(int SQ) { return SQ == 0 ? 4 : (SQ == 3 ? 1 : 2); }
__host__ __device__ constexpr int sq_row(int SQ, int r) {
    // slot 0 = V, 1 = H, 2 = E, 3 = C.  SQ 0: V->0 H->1 E->3 C->4; SQ 1: V->2 E->5; SQ 2: V->6 H->7; SQ 3: V->8
    return SQ == 0 ? (r == 0 ? 0 : r == 1 ? 1 : r == 2 ? 3 : 4)
         : SQ == 1 ? (r == 0 ? 2 : 5)
         : SQ == 2 ? (r == 0 ? 6 : 7)
                   : 8;
}
__host__ __device__ constexpr int sq_slot(int SQ, int r) {
    return SQ == 0 ? r : SQ == 1 ? (r == 0 ? 0 : 2) : SQ == 2 ? (r == 0 ? 0 : 1) : 0;
}

template <typename T>
struct Acc {
    T au[2][4];   // (A u) at the owned velocity nodes V, H, E, C
    T bt[2][4];   // (B^T p)
    T idg[4];     // 1 / diag A
    T bu;         // (B u) at the owned vertex
};

// Programmatic dependent launch: when the kernels of a cycle are launched with programmatic stream
// serialisation (pdl_enabled), a kernel's CTAs can be scheduled before its predecessor has
// finished.  Each kernel waits (pdl_wait) until every predecessor has completed and its memory is
// visible before it touches global memory, and lets its successor launch (pdl_trigger) only at its
// end, so that early-launched CTAs overlap the predecessor's tail instead of holding SM slots for
// its whole run.  Without the launch attribute both instructions return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Programmatic dependent launch unless the environment sets STOKES_MG_PDL=0 (read once per
// process).  Measured on GB300 with the trigger at the end of each kernel: 0.705 against
// 0.726 ms per refinement step at k = 8 and 84 against 86 ms for six concurrent solves; with the
// trigger at the start (successors' CTAs waiting on SMs for the whole predecessor) it had cost
// 130 against 90 ms.
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Views map P2-lattice points to values.  A velocity view answers at(si, sj, a, b), the value at
// lattice point (2 si + a, 2 sj + b) (a, b are compile-time in every caller, so a square's nine
// loads share one address computation), and (X, Y) for a single point.  A vertex view answers
// (i, j).  GView reads global memory through the read-only path; SLat / SVert read shared tiles.
template <typename T>
struct GView {
    static constexpr bool zero_filled = false;   // reads outside the array are not allowed
    const T* p;
    int ld;
    // 32-bit offsets: one array holds at most (2N+1)^2 < 2^31 values for every supported level
    __device__ __forceinline__ T operator()(int X, int Y) const { return __ldg(p + (Y * ld + X)); }
    __device__ __forceinline__ T at(int si, int sj, int a, int b) const {
        return __ldg(p + ((2 * sj + b) * ld + 2 * si + a));
    }
};
template <typename T>
__device__ __forceinline__ GView<T> gview(const T* p, int ld) { return GView<T>{p, ld}; }

// The same reads without any test: only for cells whose 5 x 5 lattice window and 3 x 3 vertex
// window lie inside the arrays (block_interior).  Declared zero-filled, so the row code neither
// tests the range nor masks the Dirichlet ring; with margin 2 no window reaches the ring at all.
template <typename T>
struct GViewU {
    static constexpr bool zero_filled = true;
    const T* p;
    int ld;
    __device__ __forceinline__ T operator()(int X, int Y) const { return __ldg(p + (Y * ld + X)); }
    __device__ __forceinline__ T at(int si, int sj, int a, int b) const {
        return __ldg(p + ((2 * sj + b) * ld + 2 * si + a));
    }
};
template <typename T>
__device__ __forceinline__ GViewU<T> gviewu(const T* p, int ld) { return GViewU<T>{p, ld}; }

// One component of a planar float32 velocity array (common.cuh, pl_u), through the read-only path:
// p is the array plus the component (0 or 1), rs and ps the row and plane strides in floats.
// ZF as for GViewU (true only where every window lies inside the lattice and off the ring).
template <bool ZF>
struct GViewP {
    static constexpr bool zero_filled = ZF;
    const float* p;
    int rs, ps;
    __device__ __forceinline__ float operator()(int X, int Y) const {
        return __ldg(p + ((X & 1) * ps + Y * rs + (X >> 1) * 2));
    }
    __device__ __forceinline__ float at(int si, int sj, int a, int b) const {
        return __ldg(p + ((a & 1) * ps + (2 * sj + b) * rs + 2 * (si + (a >> 1))));
    }
};
template <bool ZF>
__device__ __forceinline__ GViewP<ZF> gviewp(const float* u, int n, int comp) {
    const int rs = 2 * pl_pitch(n);
    return GViewP<ZF>{u + comp, rs, rs * pl_rows(n)};
}

// True when every cell (i, j) of this block has m <= i, j <= n - m (block-uniform).  Margin 1: the
// windows stay inside the arrays; margin 2: they also avoid the Dirichlet ring.
__device__ __forceinline__ bool block_interior(int n, int m) {
    const int i0 = blockIdx.x * blockDim.x, j0 = blockIdx.y * blockDim.y;
    return i0 >= m && j0 >= m && i0 + (int)blockDim.x - 1 <= n - m && j0 + (int)blockDim.y - 1 <= n - m;
}

// Shared-memory lattice tile split by the parity of X: plane (X - 2 xh0) & 1 holds the points of
// that parity, so a warp reading one local node of 32 consecutive squares touches 32 consecutive
// words.  WH words per row, PL words per plane (padded so the two planes fall on different banks).
template <typename T, int WH, int PL>
struct SLat {
    static constexpr bool zero_filled = true;    // the tile covers every window and holds 0 off the domain
    const T* p;
    int xh0, y0;   // tile origin: X0 = 2 xh0, Y0 = y0
    __device__ __forceinline__ T at(int si, int sj, int a, int b) const {
        return p[(a & 1) * PL + (2 * sj + b - y0) * WH + (si - xh0) + (a >> 1)];
    }
    __device__ __forceinline__ T operator()(int X, int Y) const {
        const int dx = X - 2 * xh0;
        return p[(dx & 1) * PL + (Y - y0) * WH + (dx >> 1)];
    }
};
template <typename T, int LD>
struct SVert {
    static constexpr bool zero_filled = true;
    const T* p;
    int x0, y0;
    __device__ __forceinline__ T operator()(int i, int j) const { return p[(j - y0) * LD + (i - x0)]; }
};

template <bool MASK, typename T, typename V>
__device__ __forceinline__ void load_sq(const V& u, int n, int si, int sj, T (&v)[9]) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T val = u.at(si, sj, a, b);
            if (MASK && !interior2(2 * si + a, 2 * sj + b, n)) val = T(0);
            v[3 * b + a] = val;
        }
}

template <typename T, typename V>
__device__ __forceinline__ void load_sq_p(const V& p, int si, int sj, T (&q)[4]) {
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) q[2 * b + a] = p(si + a, sj + b);
}

template <bool DA, bool DBT, bool DD, int O, int SQ, int R, typename T>
__device__ __forceinline__ void sq_rows(const T (&A)[2][9][9], const OpCoef<T>& c, const T (&vx)[9],
                                        const T (&vy)[9], const T (&pq)[4], Acc<T>& a) {
    if constexpr (R < sq_nrows(SQ)) {
        constexpr int L = sq_row(SQ, R), s = sq_slot(SQ, R);
        if constexpr (DA) {
            a.au[0][s] += arow<O, L>(A, vx);
            a.au[1][s] += arow<O, L>(A, vy);
        }
        if constexpr (DBT) {
            a.bt[0][s] += btrow<O, L>(c.Bx, pq);
            a.bt[1][s] += btrow<O, L>(c.By, pq);
        }
        if constexpr (DD) a.idg[s] += A[O][L][L];   // the diagonal; inverted in cell_apply
        sq_rows<DA, DBT, DD, O, SQ, R + 1>(A, c, vx, vy, pq, a);
    }
}

template <bool DA, bool DBT, bool DB, bool DD, bool MASK, int SQ, typename T, typename VU, typename VP>
__device__ __forceinline__ void visit(int i, int j, int n, const T (&A)[2][9][9], const OpCoef<T>& c,
                                      const VU& ux, const VU& uy, const VP& p, Acc<T>& a) {
    const int si = i - (SQ & 1), sj = j - (SQ >> 1);
    if (si < 0 || sj < 0 || si >= n || sj >= n) return;
    T vx[9], vy[9], pq[4];
    if constexpr (DA || DB) {
        load_sq<MASK>(ux, n, si, sj, vx);
        load_sq<MASK>(uy, n, si, sj, vy);
    }
    if constexpr (DBT) load_sq_p(p, si, sj, pq);
    if (orient(si, sj, n)) {
        sq_rows<DA, DBT, DD, 1, SQ, 0>(A, c, vx, vy, pq, a);
        if constexpr (DB) a.bu += brow<1, SQ>(c.Bx, vx) + brow<1, SQ>(c.By, vy);
    } else {
        sq_rows<DA, DBT, DD, 0, SQ, 0>(A, c, vx, vy, pq, a);
        if constexpr (DB) a.bu += brow<0, SQ>(c.Bx, vx) + brow<0, SQ>(c.By, vy);
    }
}

template <bool DA, bool DBT, bool DB, bool DD, bool MASK, typename T, typename VU, typename VP>
__device__ __forceinline__ void cell_apply(int i, int j, int n, const T (&A)[2][9][9], const OpCoef<T>& c,
                                           const VU& ux, const VU& uy, const VP& p, Acc<T>& a) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a.au[0][s] = a.au[1][s] = a.bt[0][s] = a.bt[1][s] = a.idg[s] = T(0);
    }
    a.bu = T(0);
    visit<DA, DBT, DB, DD, MASK, 0>(i, j, n, A, c, ux, uy, p, a);
    visit<DA, DBT, DB, DD, MASK, 1>(i, j, n, A, c, ux, uy, p, a);
    visit<DA, DBT, DB, DD, MASK, 2>(i, j, n, A, c, ux, uy, p, a);
    visit<DA, DBT, DB, DD, MASK, 3>(i, j, n, A, c, ux, uy, p, a);
    if constexpr (DD) {
#pragma unroll
        for (int s = 0; s < 4; ++s) a.idg[s] = T(1) / a.idg[s];   // nodes without squares: inf, never used
    }
}

// ---- merged node stencils: the rows of a cell's nodes summed over its four squares, per stencil
// class (common.cuh).  Every structural-zero test below is a template argument (the class C), so
// it is decided at compile time.
__host__ __device__ constexpr bool need_win(int C, bool DA, bool DB, int w) {
    return (DA && (nz_MA(C, 0, w) || nz_MA(C, 1, w) || nz_MA(C, 2, w) || nz_MA(C, 3, w))) || (DB && nz_MB(C, w));
}
__host__ __device__ constexpr bool need_vwin(int C, int v) {
    return nz_MBT(C, 0, v) || nz_MBT(C, 1, v) || nz_MBT(C, 2, v) || nz_MBT(C, 3, v);
}

template <int C, bool DA, bool DB, bool MASK, int W, typename T, typename VU>
__device__ __forceinline__ void win_load1(int i, int j, int n, const VU& ux, const VU& uy, T (&wx)[25], T (&wy)[25]) {
    if constexpr (need_win(C, DA, DB, W)) {
        constexpr int dx = W % 5 - 2, dy = W / 5 - 2;
        if constexpr (VU::zero_filled && !MASK) {
            wx[W] = ux.at(i - 1, j - 1, dx + 2, dy + 2);
            wy[W] = uy.at(i - 1, j - 1, dx + 2, dy + 2);
        } else {
            const int X = 2 * i + dx, Y = 2 * j + dy;
            const bool ok = MASK ? interior2(X, Y, n) : (X >= 0 && Y >= 0 && X <= 2 * n && Y <= 2 * n);
            wx[W] = ok ? ux.at(i - 1, j - 1, dx + 2, dy + 2) : T(0);
            wy[W] = ok ? uy.at(i - 1, j - 1, dx + 2, dy + 2) : T(0);
        }
    }
}
template <int C, bool DA, bool DB, bool MASK, typename T, typename VU, int... W>
__device__ __forceinline__ void win_load(int i, int j, int n, const VU& ux, const VU& uy, T (&wx)[25], T (&wy)[25],
                                         std::integer_sequence<int, W...>) {
    (win_load1<C, DA, DB, MASK, W>(i, j, n, ux, uy, wx, wy), ...);
}

template <int C, int V, typename T, typename VP>
__device__ __forceinline__ void vwin_load1(int i, int j, int n, const VP& p, T (&pw)[9]) {
    if constexpr (need_vwin(C, V)) {
        const int I = i + V % 3 - 1, J = j + V / 3 - 1;
        if constexpr (VP::zero_filled) pw[V] = p(I, J);
        else pw[V] = (I >= 0 && J >= 0 && I <= n && J <= n) ? p(I, J) : T(0);
    }
}
template <int C, typename T, typename VP, int... V>
__device__ __forceinline__ void vwin_load(int i, int j, int n, const VP& p, T (&pw)[9], std::integer_sequence<int, V...>) {
    (vwin_load1<C, V>(i, j, n, p, pw), ...);
}

template <int C, int S, int K, typename T>
__device__ __forceinline__ void ma_term(const OpCoef<T>& c, const T (&w)[25], T& s) {
    if constexpr (nz_MA(C, S, K)) s = fma(c.MA[C][S][K], w[K], s);
}
template <int C, int S, typename T, int... K>
__device__ __forceinline__ T ma_row_i(const OpCoef<T>& c, const T (&w)[25], std::integer_sequence<int, K...>) {
    T s = T(0);
    (ma_term<C, S, K>(c, w, s), ...);
    return s;
}
template <int C, int S, typename T>
__device__ __forceinline__ T ma_row(const OpCoef<T>& c, const T (&w)[25]) {
    return ma_row_i<C, S>(c, w, std::make_integer_sequence<int, 25>{});
}

template <int C, int S, int K, typename T>
__device__ __forceinline__ void mbt_term(const T (&B)[kStencilClasses][4][9], const T (&pw)[9], T& s) {
    if constexpr (nz_MBT(C, S, K)) s = fma(B[C][S][K], pw[K], s);
}
template <int C, int S, typename T, int... K>
__device__ __forceinline__ T mbt_row_i(const T (&B)[kStencilClasses][4][9], const T (&pw)[9],
                                       std::integer_sequence<int, K...>) {
    T s = T(0);
    (mbt_term<C, S, K>(B, pw, s), ...);
    return s;
}
template <int C, int S, typename T>
__device__ __forceinline__ T mbt_row(const T (&B)[kStencilClasses][4][9], const T (&pw)[9]) {
    return mbt_row_i<C, S>(B, pw, std::make_integer_sequence<int, 9>{});
}

template <int C, int K, typename T>
__device__ __forceinline__ void mb_term(const OpCoef<T>& c, const T (&wx)[25], const T (&wy)[25], T& s) {
    if constexpr (nz_MB(C, K)) s = fma(c.MBx[C][K], wx[K], fma(c.MBy[C][K], wy[K], s));
}
template <int C, typename T, int... K>
__device__ __forceinline__ T mb_row_i(const OpCoef<T>& c, const T (&wx)[25], const T (&wy)[25],
                                      std::integer_sequence<int, K...>) {
    T s = T(0);
    (mb_term<C, K>(c, wx, wy, s), ...);
    return s;
}

template <bool DA, bool DBT, bool DB, bool DD, bool MASK, int C, typename T, typename VU, typename VP>
__device__ __forceinline__ void cell_apply_merged(int i, int j, int n, const OpCoef<T>& c, const VU& ux, const VU& uy,
                                                  const VP& p, Acc<T>& a) {
    T wx[25], wy[25], pw[9];
    if constexpr (DA || DB) win_load<C, DA, DB, MASK>(i, j, n, ux, uy, wx, wy, std::make_integer_sequence<int, 25>{});
    if constexpr (DBT) vwin_load<C>(i, j, n, p, pw, std::make_integer_sequence<int, 9>{});
#pragma unroll
    for (int s = 0; s < 4; ++s) a.au[0][s] = a.au[1][s] = a.bt[0][s] = a.bt[1][s] = a.idg[s] = T(0);
    a.bu = T(0);
    if constexpr (DA) {
        a.au[0][0] = ma_row<C, 0>(c, wx); a.au[1][0] = ma_row<C, 0>(c, wy);
        a.au[0][1] = ma_row<C, 1>(c, wx); a.au[1][1] = ma_row<C, 1>(c, wy);
        a.au[0][2] = ma_row<C, 2>(c, wx); a.au[1][2] = ma_row<C, 2>(c, wy);
        a.au[0][3] = ma_row<C, 3>(c, wx); a.au[1][3] = ma_row<C, 3>(c, wy);
    }
    if constexpr (DBT) {
        a.bt[0][0] = mbt_row<C, 0>(c.MBTx, pw); a.bt[1][0] = mbt_row<C, 0>(c.MBTy, pw);
        a.bt[0][1] = mbt_row<C, 1>(c.MBTx, pw); a.bt[1][1] = mbt_row<C, 1>(c.MBTy, pw);
        a.bt[0][2] = mbt_row<C, 2>(c.MBTx, pw); a.bt[1][2] = mbt_row<C, 2>(c.MBTy, pw);
        a.bt[0][3] = mbt_row<C, 3>(c.MBTx, pw); a.bt[1][3] = mbt_row<C, 3>(c.MBTy, pw);
    }
    if constexpr (DD) {
#pragma unroll
        for (int s = 0; s < 4; ++s) a.idg[s] = c.MIdg[C][s];
    }
    if constexpr (DB) a.bu = mb_row_i<C>(c, wx, wy, std::make_integer_sequence<int, 25>{});
}

// Operator rows of cell (i, j) from the merged stencils of its class (branch uniform across a warp
// except where the warp meets a mid-line).
template <bool DA, bool DBT, bool DB, bool DD, bool MASK, typename T, typename VU, typename VP>
__device__ __forceinline__ void cell_apply_auto(int i, int j, int n, const OpCoef<T>& c, const VU& ux, const VU& uy,
                                                const VP& p, Acc<T>& a) {
    switch (stencil_class(i, j, n)) {
        case 0: cell_apply_merged<DA, DBT, DB, DD, MASK, 0>(i, j, n, c, ux, uy, p, a); break;
        case 1: cell_apply_merged<DA, DBT, DB, DD, MASK, 1>(i, j, n, c, ux, uy, p, a); break;
        case 2: cell_apply_merged<DA, DBT, DB, DD, MASK, 2>(i, j, n, c, ux, uy, p, a); break;
        case 3: cell_apply_merged<DA, DBT, DB, DD, MASK, 3>(i, j, n, c, ux, uy, p, a); break;
        case 4: cell_apply_merged<DA, DBT, DB, DD, MASK, 4>(i, j, n, c, ux, uy, p, a); break;
        case 5: cell_apply_merged<DA, DBT, DB, DD, MASK, 5>(i, j, n, c, ux, uy, p, a); break;
        default: cell_apply_merged<DA, DBT, DB, DD, MASK, 6>(i, j, n, c, ux, uy, p, a); break;
    }
}

// lattice position and existence / unknown flags of slot s of cell (i, j)
__device__ __forceinline__ void slot_pos(int i, int j, int s, int& X, int& Y) {
    X = 2 * i + (s & 1);
    Y = 2 * j + (s >> 1);
}
__device__ __forceinline__ bool slot_exists(const CellNodes& cn, int s) {
    return s == 0 ? true : s == 1 ? cn.hx : s == 2 ? cn.ex : cn.cx;
}
__device__ __forceinline__ bool slot_unknown(const CellNodes& cn, int s) {
    return s == 0 ? cn.v : s == 1 ? cn.h : s == 2 ? cn.e : cn.c;
}

// (kernels that reduce over the block with block_sum2d are launched with BX x BY threads)
#define CELL_INDEX                                          \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;    \
    const int j = blockIdx.y * blockDim.y + threadIdx.y;    \
    const bool active = i <= n && j <= n;                   \
    const int tid = threadIdx.y * blockDim.x + threadIdx.x; \
    (void)tid;

// Block sums of two doubles at once (one barrier); results valid in tid 0.
__device__ __forceinline__ double2 block_sum2d_pair(double a, double b, int tid) {
    __shared__ double2 red2[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((tid & 31) == 0) red2[tid >> 5] = make_double2(a, b);
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (tid < 32) {
        s = tid < NT / 32 ? red2[tid] : make_double2(0.0, 0.0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_down_sync(0xffffffffu, s.x, o);
            s.y += __shfl_down_sync(0xffffffffu, s.y, o);
        }
    }
    return s;
}

// Block sums of a float (summed in float: a sum of squares for a convergence test) and a double
// (one barrier); results valid in tid 0.  Keeps the second sum off the float64 pipe.
__device__ __forceinline__ double2 block_sum2_fd(float a, double b, int tid) {
    __shared__ float redf[NT / 32];
    __shared__ double redd[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((tid & 31) == 0) {
        redf[tid >> 5] = a;
        redd[tid >> 5] = b;
    }
    __syncthreads();
    float sa = 0.f;
    double sb = 0.0;
    if (tid < 32) {
        sa = tid < NT / 32 ? redf[tid] : 0.f;
        sb = tid < NT / 32 ? redd[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_down_sync(0xffffffffu, sa, o);
            sb += __shfl_down_sync(0xffffffffu, sb, o);
        }
    }
    return make_double2((double)sa, sb);
}

// Block sum (thread-linear id tid) of one double; result valid in tid 0.
__device__ __forceinline__ double block_sum2d(double v, int tid) {
    __shared__ double red[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid < 32) {
        s = tid < NT / 32 ? red[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}


}  // namespace smg
