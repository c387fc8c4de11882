// uzawa_reg.cu -- the float32 Uzawa step (Sec. 4) in one kernel with the operator's coefficients
// held in registers.
//
//   u^{m-1/2} = u^{m-1} + tau Ahat^{-1} (f - A u^{m-1} - B^T p^{m-1})
//   dp        = sigma Shat^{-1} (B u^{m-1/2} - g),      p^{m} = p^{m-1} + dp
//   u^{m}     = u^{m-1/2} - tau Ahat^{-1} B^T dp
//
// Away from the two mid-lines every cell has the stencils of its quadrant's orientation class, and
// these stencils are far sparser and more regular than their structural pattern: the four velocity
// rows of a cell (V, H, E, C) have 17 + 9 + 9 + 7 nonzero coefficients (for every beta and h: K has
// the zero couplings of the P2 stiffness on right isosceles triangles, M those of the P2 mass), which
// take only eight distinct values per class (the mesh's point and diagonal symmetries and A = A^T);
// the vertex row of B^T vanishes, and every entry of B and B^T is +-b or +-b/2 for one b ~ h.  The
// kernel therefore keeps the eight A values as (a, a) pairs in sixteen registers, applies each A
// term with one packed FP32x2 FMA on the (u_x, u_y) pair, and forms B u and B^T p as sums with the
// literal weights +-1, +-1/2, scaled once by b.  The structure is a compile-time table (below),
// checked against the level's assembled coefficients on the host before every launch
// (make_reg_coef).
//
// Data movement: a CTA owns a 28 x ty tile of cells and stages, with asynchronous 4-byte copies
// (cp.async, zero-filled off the domain), u with a three-cell halo as (u_x, u_y) pairs split by the
// parity of the lattice column, p with the same halo, f on the tile plus two cells, and g, Shat^{-1}
// on the tile plus one vertex.  u^{m-1/2} overwrites f in place (each value read and written by the
// same thread) and dp overwrites g.  Tiles whose u^{m-1/2} region meets a mid-line take the general
// per-cell rows of cellops.cuh on the same shared tiles.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cuda.h>

#include "cellops.cuh"
#include "elements.h"
#include "kernels.cuh"
#include "tiles.cuh"

namespace smg {
namespace {

// ---------------------------------------------------------------------------------------------
// Structure of the merged stencils of the orientation classes 0 and 1 (common.cuh), by window
// point w = (dy + 2) * 5 + dx + 2 of the 5 x 5 lattice window around the cell's vertex (2i, 2j)
// and owned node s (0 V, 1 H, 2 E, 3 C):
//   kGid[cls][s][w]  group of the A coefficient (-1: zero); every group holds one value
//   kBx / kBy[cls][w]  the vertex's B row in units of b/2 (values 0, +-1, +-2)
//   kBTx / kBTy[cls][s][v]  the B^T rows over the 3 x 3 vertex window v = (dj + 1) * 3 + di + 1,
//                           in units of b/2
constexpr int kGroups = 8;
constexpr int kGidDiagV = 4, kGidDiagE = 7;   // groups of the diagonal of the V row and of the H, E, C rows
constexpr signed char kGid[2][4][25] = {
    {{0, 1, 2, -1, -1, 1, -1, 3, 1, -1, 2, 3, 4, 3, 2, -1, 1, 3, -1, 1, -1, -1, 2, 1, 0},
     {-1, -1, 1, -1, -1, -1, -1, 5, 6, -1, -1, -1, 3, 7, 3, -1, -1, -1, 6, 5, -1, -1, -1, -1, 1},
     {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 1, 5, 3, -1, -1, -1, 6, 7, 6, -1, -1, -1, 3, 5, 1},
     {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 6, 1, -1, -1, 6, 7, 6, -1, -1, 1, 6, -1}},
    {{-1, -1, 0, 1, 2, -1, 1, 3, -1, 1, 0, 3, 4, 3, 0, 1, -1, 3, 1, -1, 2, 1, 0, -1, -1},
     {-1, -1, -1, -1, 1, -1, -1, -1, 5, 6, -1, -1, 3, 7, 3, -1, -1, 6, 5, -1, -1, -1, 1, -1, -1},
     {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 3, 6, 1, -1, 5, 7, 5, -1, 1, 6, 3, -1, -1},
     {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 1, 5, -1, -1, -1, 5, 7, 5, -1, -1, -1, 5, 1}}};
constexpr signed char kBx[2][25] = {
    {0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, -2, 0, 2, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, -2, 0, 2, 0, -1, -1, 1, 1, 0, 0, 0, 0, 0, 0}};
constexpr signed char kBy[2][25] = {
    {0, -1, 0, 0, 0, 0, -1, -2, -1, 0, 0, 1, 0, -1, 0, 0, 1, 2, 1, 0, 0, 0, 0, 1, 0},
    {0, 0, 0, -1, 0, 0, -1, -2, -1, 0, 0, -1, 0, 1, 0, 0, 1, 2, 1, 0, 0, 1, 0, 0, 0}};
constexpr signed char kBTx[2][4][9] = {
    {{0, 0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 2, -2, 0, 0, 0}, {0, 0, 0, 1, -1, 0, 0, 1, -1}, {0, 0, 0, 0, 1, -1, 0, 1, -1}},
    {{0, 0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 2, -2, 0, 0, 0}, {0, 0, 0, 0, 1, -1, 1, -1, 0}, {0, 0, 0, 0, 1, -1, 0, 1, -1}}};
constexpr signed char kBTy[2][4][9] = {
    {{0, 0, 0, 0, 0, 0, 0, 0, 0}, {0, 1, 0, 0, -1, 1, 0, 0, -1}, {0, 0, 0, 0, 2, 0, 0, -2, 0}, {0, 0, 0, 0, 1, 1, 0, -1, -1}},
    {{0, 0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 1, 0, 1, -1, 0, -1, 0}, {0, 0, 0, 0, 2, 0, 0, -2, 0}, {0, 0, 0, 0, 1, 1, 0, -1, -1}}};

__host__ __device__ constexpr bool a_win(int C, int w) {
    return kGid[C][0][w] >= 0 || kGid[C][1][w] >= 0 || kGid[C][2][w] >= 0 || kGid[C][3][w] >= 0;
}
__host__ __device__ constexpr bool bt_vwin(int C, int v) {
    for (int s = 0; s < 4; ++s)
        if (kBTx[C][s][v] != 0 || kBTy[C][s][v] != 0) return true;
    return false;
}

}  // namespace

// Values of the structure above for one level (host-built by make_reg_coef)
struct RegCoef {
    float2 a[2][kGroups];   // A group values as (a, a) pairs, per class
    float ti[2][2];         // tau / diag A: [class][0 = V row, 1 = H, E, C rows]
    float b;                // B = (b / 2) x (the integer tables)
};

// Fills q from the level's merged stencils and checks that they have exactly the compile-time
// structure (zeros, equal groups, B entries +-b, +-b/2); false if not (the caller then uses
// another step variant).
static bool make_reg_coef(const OpCoef<float>& c, float tau, RegCoef& q) {
    double amax = 0.0, bmax = 0.0;
    for (int C = 0; C < 2; ++C) {
        for (int s = 0; s < 4; ++s)
            for (int w = 0; w < 25; ++w) amax = std::max(amax, std::fabs((double)c.MA[C][s][w]));
        for (int w = 0; w < 25; ++w) bmax = std::max({bmax, std::fabs((double)c.MBx[C][w]), std::fabs((double)c.MBy[C][w])});
    }
    if (!(amax > 0.0) || !(bmax > 0.0)) return false;
    const double b = bmax;
    for (int C = 0; C < 2; ++C) {
        bool set[kGroups] = {};
        for (int s = 0; s < 4; ++s)
            for (int w = 0; w < 25; ++w) {
                const double v = c.MA[C][s][w];
                const int gid = kGid[C][s][w];
                if (gid < 0) {
                    if (std::fabs(v) > 1e-6 * amax) return false;
                    continue;
                }
                if (!set[gid]) {
                    q.a[C][gid] = make_float2((float)v, (float)v);
                    set[gid] = true;
                } else if (std::fabs(v - (double)q.a[C][gid].x) > 1e-6 * std::fabs(v) + 1e-7 * amax) {
                    return false;
                }
            }
        for (int g = 0; g < kGroups; ++g)
            if (!set[g]) return false;
        for (int w = 0; w < 25; ++w)
            if (std::fabs(c.MBx[C][w] - 0.5 * b * kBx[C][w]) > 1e-6 * b ||
                std::fabs(c.MBy[C][w] - 0.5 * b * kBy[C][w]) > 1e-6 * b)
                return false;
        for (int s = 0; s < 4; ++s)
            for (int v = 0; v < 9; ++v)
                if (std::fabs(c.MBTx[C][s][v] - 0.5 * b * kBTx[C][s][v]) > 1e-6 * b ||
                    std::fabs(c.MBTy[C][s][v] - 0.5 * b * kBTy[C][s][v]) > 1e-6 * b)
                    return false;
        // the diagonal groups are the stored inverse diagonals
        if (std::fabs(1.0 / q.a[C][kGidDiagV].x - c.MIdg[C][0]) > 1e-6 * std::fabs(c.MIdg[C][0])) return false;
        for (int s = 1; s < 4; ++s)
            if (std::fabs(1.0 / q.a[C][kGidDiagE].x - c.MIdg[C][s]) > 1e-6 * std::fabs(c.MIdg[C][s])) return false;
        q.ti[C][0] = tau * c.MIdg[C][0];
        q.ti[C][1] = tau * c.MIdg[C][1];
    }
    q.b = (float)b;
    return true;
}

bool reg_tables_match(const OpCoef<float>& c) {
    RegCoef q;
    return make_reg_coef(c, 1.0f, q);
}

namespace {

// Shared-memory tile geometry.  A CTA owns cells [i0, i0 + TX) x [j0, j0 + ty).  The u tile holds
// cells from i0 - UX (two planes by column parity, UWH (u_x, u_y) pairs per lattice row, rows from
// 2 (j0 - 3)); the f / u^{m-1/2} tile cells [i0 - 2, i0 + TX + 2) x [j0 - 2, j0 + ty + 2) (four planes
// by node type, FW pairs per row); the p tile vertices from (i0 - PX, j0 - 3), PW per row; the g,
// Shat^{-1} and dp tiles vertices from (i0 - DX, j0 - 1), DW per row, of which DN are computed.
struct RegTile {   // staged by 4-byte asynchronous copies from the compact float32 layout
    static constexpr int TX = 28;
    static_assert(TX + 4 == 32, "one warp covers a row of the u^{m-1/2} region");
    static constexpr int UX = 3, PX = 3, DX = 1;
    static constexpr int UWH = TX + 6;   // u: cells [i0-3, i0+TX+3); float2 per parity-plane row
    static constexpr int PW = TX + 6;    // p: vertices [i0-3, i0+TX+3)
    static constexpr int FW = TX + 4;    // f, u^{m-1/2}: cells [i0-2, i0+TX+2), one plane per node type
    static constexpr int DW = TX + 2;    // g, Shat^{-1}, dp: vertices [i0-1, i0+TX+1)
    static constexpr int DN = TX + 2;
    // planes are padded to 8 float2 modulo 16 so that two planes start 16 banks apart: a warp that
    // stages 16 consecutive lattice points (both components) writes 32 distinct banks
    __host__ __device__ static constexpr int pad8(int m) { return m + ((8 - m % 16) + 16) % 16; }
    __host__ __device__ static constexpr int upl(int ty) { return pad8(UWH * 2 * (ty + 6)); }   // float2 per u plane
    __host__ __device__ static constexpr int fpl(int ty) { return pad8(FW * (ty + 4)); }        // float2 per f plane
    __host__ __device__ static constexpr int dsz(int ty) { return DW * (ty + 2); }
    __host__ __device__ static constexpr size_t bytes(int ty) {
        return 8 * (size_t)(2 * upl(ty) + 4 * fpl(ty)) + 4 * (size_t)(PW * (ty + 6) + 2 * dsz(ty));
    }
};

// The same tile staged by the tensor-memory-access engine from the planar float32 layout: each tile
// is one box copy, so rows start on 16-byte boundaries (the u and vertex tiles start one cell or
// vertex further left, at a multiple of 4) and planes are dense.  Buffers are 128-byte aligned after
// a 128-byte slot for the mbarrier.
struct TmaTile {
    static constexpr int TX = 28;
    static constexpr int UX = 4, PX = 4, DX = 4;
    static constexpr int UWH = 36;       // u: pairs [i0-4, i0+32)
    static constexpr int PW = 36;        // p: vertices [i0-4, i0+32)
    static constexpr int FW = TX + 4;
    static constexpr int DW = 36;        // g, Shat^{-1}, dp: vertices [i0-4, i0+32)
    static constexpr int DN = TX + 2;
    __host__ __device__ static constexpr int upl(int ty) { return UWH * 2 * (ty + 6); }
    __host__ __device__ static constexpr int fpl(int ty) { return FW * (ty + 4); }
    __host__ __device__ static constexpr int dsz(int ty) { return DW * (ty + 2); }
    __host__ __device__ static constexpr size_t a128(size_t b) { return (b + 127) / 128 * 128; }
    __host__ __device__ static constexpr size_t off_f(int ty) { return 128 + a128(8 * (size_t)(2 * upl(ty))); }
    __host__ __device__ static constexpr size_t off_p(int ty) { return off_f(ty) + a128(8 * (size_t)(4 * fpl(ty))); }
    __host__ __device__ static constexpr size_t off_g(int ty) { return off_p(ty) + a128(4 * (size_t)(PW * (ty + 6))); }
    __host__ __device__ static constexpr size_t off_s(int ty) { return off_g(ty) + a128(4 * (size_t)dsz(ty)); }
    // dynamic shared memory per CTA (plus 128 bytes to align the base)
    __host__ __device__ static constexpr size_t bytes(int ty) { return off_s(ty) + a128(4 * (size_t)dsz(ty)) + 128; }
    // bytes the copies of one tile deliver
    __host__ __device__ static constexpr unsigned tx_bytes(int ty) {
        return (unsigned)(8 * (2 * upl(ty) + 4 * fpl(ty)) + 4 * (PW * (ty + 6) + 2 * dsz(ty)));
    }
};
constexpr int kRegMaxRows = 24;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// 4-byte asynchronous copy global -> shared, zero-filled when !valid (the source is then not read)
__device__ __forceinline__ void cp4(void* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit_wait() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// One component of the f / u^{m-1/2} tile (four planes by node type, FW float2 per row); lattice
// coordinates are absolute, the region starts at cell (xc0, yc0).
template <class G>
struct QuadLat {
    static constexpr bool zero_filled = true;
    const float2* p;
    int pl, xc0, yc0;
    bool ycomp;
    __device__ __forceinline__ float operator()(int X, int Y) const {
        const int dx = X - 2 * xc0, dy = Y - 2 * yc0;
        const float2 e = p[((dx & 1) + 2 * (dy & 1)) * pl + (dy >> 1) * G::FW + (dx >> 1)];
        return ycomp ? e.y : e.x;
    }
    __device__ __forceinline__ float at(int si, int sj, int a, int b) const { return (*this)(2 * si + a, 2 * sj + b); }
};
// one component of the u tile (two planes by column parity, as in uzawa_pair.cu)
template <class G>
struct ULat {
    static constexpr bool zero_filled = true;
    const float2* p;
    int pl, xh0, y0;
    bool ycomp;
    __device__ __forceinline__ float at(int si, int sj, int a, int b) const {
        const float2 e = p[(a & 1) * pl + (2 * sj + b - y0) * G::UWH + (si - xh0) + (a >> 1)];
        return ycomp ? e.y : e.x;
    }
    __device__ __forceinline__ float operator()(int X, int Y) const {
        const int dx = X - 2 * xh0;
        const float2 e = p[(dx & 1) * pl + (Y - y0) * G::UWH + (dx >> 1)];
        return ycomp ? e.y : e.x;
    }
};

// acc += (k / 2) v with a compile-time k in {0, +-1, +-2}
template <int K>
__device__ __forceinline__ void addk(float& acc, float v) {
    if constexpr (K == 2) acc += v;
    else if constexpr (K == -2) acc -= v;
    else if constexpr (K == 1) acc = fmaf(0.5f, v, acc);
    else if constexpr (K == -1) acc = fmaf(-0.5f, v, acc);
}

// ---- phase 1, fast path: A rows over the u window, B^T rows over the p window
template <int C, int UWH, int W>
__device__ __forceinline__ void a_term(const float2 (&a)[kGroups], const float2* t0, const float2* t1, float2 (&au)[4],
                                       float2 (&ctr)[4]) {
    if constexpr (a_win(C, W)) {
        constexpr int dx = W % 5 - 2, dy = W / 5 - 2;
        constexpr int g0 = kGid[C][0][W], g1 = kGid[C][1][W], g2 = kGid[C][2][W], g3 = kGid[C][3][W];
        const float2 w = ((dx & 1) ? t1 : t0)[dy * UWH + (dx >> 1)];
        if constexpr (g0 >= 0) au[0] = __ffma2_rn(a[g0], w, au[0]);
        if constexpr (g1 >= 0) au[1] = __ffma2_rn(a[g1], w, au[1]);
        if constexpr (g2 >= 0) au[2] = __ffma2_rn(a[g2], w, au[2]);
        if constexpr (g3 >= 0) au[3] = __ffma2_rn(a[g3], w, au[3]);
        if constexpr (W == 12) ctr[0] = w;
        if constexpr (W == 13) ctr[1] = w;
        if constexpr (W == 17) ctr[2] = w;
        if constexpr (W == 18) ctr[3] = w;
    }
}
template <int C, int UWH, int... W>
__device__ __forceinline__ void a_rows(const float2 (&a)[kGroups], const float2* t0, const float2* t1, float2 (&au)[4],
                                       float2 (&ctr)[4], std::integer_sequence<int, W...>) {
    (a_term<C, UWH, W>(a, t0, t1, au, ctr), ...);
}
// B^T rows of the H, E, C nodes (the V row is zero) over a 3 x 3 vertex window at sp[b], row pitch LD
template <int C, int LD, int V>
__device__ __forceinline__ void bt_term(const float* sp, float2 (&bt)[4]) {
    if constexpr (bt_vwin(C, V)) {
        const float v = sp[(V / 3 - 1) * LD + V % 3 - 1];
        addk<kBTx[C][1][V]>(bt[1].x, v);
        addk<kBTy[C][1][V]>(bt[1].y, v);
        addk<kBTx[C][2][V]>(bt[2].x, v);
        addk<kBTy[C][2][V]>(bt[2].y, v);
        addk<kBTx[C][3][V]>(bt[3].x, v);
        addk<kBTy[C][3][V]>(bt[3].y, v);
    }
}
template <int C, int LD, int... V>
__device__ __forceinline__ void bt_rows(const float* sp, float2 (&bt)[4], std::integer_sequence<int, V...>) {
    (bt_term<C, LD, V>(sp, bt), ...);
}
// B row of a vertex over the u^{m-1/2} window: f0 points at the vertex's node in plane 0
template <int C, int FW, int W>
__device__ __forceinline__ void b_term(const float2* f0, int fpl, float& acc) {
    if constexpr (kBx[C][W] != 0 || kBy[C][W] != 0) {
        constexpr int dx = W % 5 - 2, dy = W / 5 - 2;
        constexpr int plane = (dx & 1) + 2 * (dy & 1);
        const float2 w = f0[plane * fpl + (dy >> 1) * FW + (dx >> 1)];
        addk<kBx[C][W]>(acc, w.x);
        addk<kBy[C][W]>(acc, w.y);
    }
}
template <int C, int FW, int... W>
__device__ __forceinline__ float b_row(const float2* f0, int fpl, std::integer_sequence<int, W...>) {
    float acc = 0.f;
    (b_term<C, FW, W>(f0, fpl, acc), ...);
    return acc;
}

template <int C>
__device__ __forceinline__ void load_coef(const RegCoef& q, float2 (&a)[kGroups]) {
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        a[g] = q.a[C][g];
        // keep the values in registers (the compiler may not rematerialise them from the constant bank)
        asm("" : "+f"(a[g].x), "+f"(a[g].y));
    }
}

template <class G, int C, bool INNER>
__device__ __forceinline__ void phase1_fast(const RegCoef& q, const float2* sU, int UPL, const float* sP, float2* sF,
                                           int FPL, int TY, int NW, int warp, int lane, int i0, int j0, int n) {
    float2 a[kGroups];
    load_coef<C>(q, a);
    const float ti0 = q.ti[C][0], ti1 = q.ti[C][1];
    const float2 mb = f2(-q.b, -q.b);
    for (int r = warp; r < TY + 4; r += NW) {
        const float2* t0 = sU + 2 * (r + 1) * G::UWH + lane + G::UX - 2;
        const float2* t1 = t0 + UPL;
        float2 au[4], ctr[4], bt[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) au[s] = ctr[s] = bt[s] = f2(0.f, 0.f);
        a_rows<C, G::UWH>(a, t0, t1, au, ctr, std::make_integer_sequence<int, 25>{});
        bt_rows<C, G::PW>(sP + (r + 1) * G::PW + lane + G::PX - 2, bt, std::make_integer_sequence<int, 9>{});
        // only unknowns keep their value (interior tiles hold nothing else)
        bool unk[4] = {true, true, true, true};
        if constexpr (!INNER) {
            const int ci = i0 - 2 + lane, cj = j0 - 2 + r;
            const bool ci_in = ci > 0 && ci < n, cj_in = cj > 0 && cj < n;
            const bool ci_h = ci >= 0 && ci < n, cj_h = cj >= 0 && cj < n;
            unk[0] = ci_in && cj_in;
            unk[1] = ci_h && cj_in;
            unk[2] = ci_in && cj_h;
            unk[3] = ci_h && cj_h;
        }
        float2* fr = sF + r * G::FW + lane;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float2 fs = fr[s * FPL];
            const float ti = s == 0 ? ti0 : ti1;
            // u^{m-1/2} = u + ti (f - A u - b (B^T p / b)); the V row of B^T is zero
            float2 t = f2(fs.x - au[s].x, fs.y - au[s].y);
            if (s > 0) t = __ffma2_rn(mb, bt[s], t);
            const float2 h = __ffma2_rn(f2(ti, ti), t, ctr[s]);
            if constexpr (INNER) fr[s * FPL] = h;
            else fr[s * FPL] = unk[s] ? h : f2(0.f, 0.f);
        }
    }
}

template <class G, int C>
__device__ __forceinline__ void phase2_fast(const RegCoef& q, const float2* sF, int FPL, float* sG, const float* sS,
                                            float sigma, int TY, int NW, int warp, int lane) {
    const float b = q.b;
    for (int r = warp; r < TY + 2; r += NW) {
        if (lane >= G::DN) break;
        const float2* f0 = sF + (r + 1) * G::FW + lane + 1;
        const float acc = b_row<C, G::FW>(f0, FPL, std::make_integer_sequence<int, 25>{});
        const int k = r * G::DW + lane + G::DX - 1;
        // Shat^{-1} is zero-filled off the domain, so dp = 0 there
        sG[k] = sigma * sS[k] * fmaf(b, acc, -sG[k]);
    }
}

// Where a cell's new values go: the compact float32 lattice (PLO false) or the planar layout
template <bool PLO>
__device__ __forceinline__ void store_node(float* __restrict__ u_out, int n, int X, int Y, float2 v) {
    if constexpr (PLO) {
        *reinterpret_cast<float2*>(u_out + pl_u(n, X, Y)) = v;
    } else {
        const int ld = 2 * n + 1, k = Y * ld + X;
        u_out[k] = v.x;
        u_out[ld * ld + k] = v.y;
    }
}
template <bool PLO>
__device__ __forceinline__ int vert_at(int n, int i, int j) {
    return j * (PLO ? pl_vpitch(n) : n + 1) + i;
}

template <class G, bool PLO, int C, bool INNER>
__device__ __forceinline__ void phase3_fast(const RegCoef& q, const float2* sF, int FPL, const float* sG,
                                            const float* sP, int TY, int NW, int warp, int lane, int i0, int j0,
                                            int n, float* __restrict__ u_out, float* __restrict__ p_out) {
    const float nb1 = -q.ti[C][1] * q.b;
    for (int r = warp; r < TY; r += NW) {
        if (lane >= G::TX) break;
        const int ci = i0 + lane, cj = j0 + r;
        if (!INNER && (ci > n || cj > n)) continue;
        float2 bt[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) bt[s] = f2(0.f, 0.f);
        bt_rows<C, G::DW>(sG + (r + 1) * G::DW + lane + G::DX, bt, std::make_integer_sequence<int, 9>{});
        const float2* hr = sF + (r + 2) * G::FW + lane + 2;
        float2 o[4];
        o[0] = hr[0];
#pragma unroll
        for (int s = 1; s < 4; ++s) o[s] = __ffma2_rn(f2(nb1, nb1), bt[s], hr[s * FPL]);
        if constexpr (INNER) {
#pragma unroll
            for (int s = 0; s < 4; ++s) store_node<PLO>(u_out, n, 2 * ci + (s & 1), 2 * cj + (s >> 1), o[s]);
        } else {
            const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!slot_exists(cn, s)) continue;
                store_node<PLO>(u_out, n, 2 * ci + (s & 1), 2 * cj + (s >> 1),
                                slot_unknown(cn, s) ? o[s] : f2(0.f, 0.f));
            }
        }
        p_out[vert_at<PLO>(n, ci, cj)] = sP[(r + 3) * G::PW + lane + G::PX] + sG[(r + 1) * G::DW + lane + G::DX];
    }
}

// ---- the same phases two cell (or vertex) rows at a time: the windows of rows r and r + 1 overlap
// in three of their five lattice rows (two of three vertex rows), so each shared value they share is
// loaded once for both (fewer shared-memory wavefronts per cell).  Needs an even tile height.

// the A group terms of window point W applied to the value w
template <int C, int W>
__device__ __forceinline__ void a_apply(const float2 (&a)[kGroups], float2 w, float2 (&au)[4], float2 (&ctr)[4]) {
    constexpr int g0 = kGid[C][0][W], g1 = kGid[C][1][W], g2 = kGid[C][2][W], g3 = kGid[C][3][W];
    if constexpr (g0 >= 0) au[0] = __ffma2_rn(a[g0], w, au[0]);
    if constexpr (g1 >= 0) au[1] = __ffma2_rn(a[g1], w, au[1]);
    if constexpr (g2 >= 0) au[2] = __ffma2_rn(a[g2], w, au[2]);
    if constexpr (g3 >= 0) au[3] = __ffma2_rn(a[g3], w, au[3]);
    if constexpr (W == 12) ctr[0] = w;
    if constexpr (W == 13) ctr[1] = w;
    if constexpr (W == 17) ctr[2] = w;
    if constexpr (W == 18) ctr[3] = w;
}
// lattice point at row offset R (-2..4 from row r's centre) and column offset DX: window point
// (R + 2) * 5 + DX + 2 of row r (A) and R * 5 + DX + 2 of row r + 1 (B)
template <int C, int UWH, int I>
__device__ __forceinline__ void a_pair_term(const float2 (&a)[kGroups], const float2* t0, const float2* t1,
                                            float2 (&auA)[4], float2 (&ctrA)[4], float2 (&auB)[4],
                                            float2 (&ctrB)[4]) {
    constexpr int R = I / 5 - 2, DX = I % 5 - 2;
    constexpr int WA = (R + 2) * 5 + DX + 2, WB = R * 5 + DX + 2;
    constexpr bool useA = R <= 2 && a_win(C, WA), useB = R >= 0 && a_win(C, WB);
    if constexpr (useA || useB) {
        const float2 w = ((DX & 1) ? t1 : t0)[R * UWH + (DX >> 1)];
        if constexpr (useA) a_apply<C, (useA ? WA : 0)>(a, w, auA, ctrA);
        if constexpr (useB) a_apply<C, (useB ? WB : 0)>(a, w, auB, ctrB);
    }
}
template <int C, int UWH, int... I>
__device__ __forceinline__ void a_pair_rows(const float2 (&a)[kGroups], const float2* t0, const float2* t1,
                                            float2 (&auA)[4], float2 (&ctrA)[4], float2 (&auB)[4], float2 (&ctrB)[4],
                                            std::integer_sequence<int, I...>) {
    (a_pair_term<C, UWH, I>(a, t0, t1, auA, ctrA, auB, ctrB), ...);
}
// B^T rows of the H, E, C nodes of window point V applied to the vertex value v
template <int C, int V>
__device__ __forceinline__ void bt_apply(float v, float2 (&bt)[4]) {
    addk<kBTx[C][1][V]>(bt[1].x, v);
    addk<kBTy[C][1][V]>(bt[1].y, v);
    addk<kBTx[C][2][V]>(bt[2].x, v);
    addk<kBTy[C][2][V]>(bt[2].y, v);
    addk<kBTx[C][3][V]>(bt[3].x, v);
    addk<kBTy[C][3][V]>(bt[3].y, v);
}
// vertex at row offset RV (-1..2 from row r's centre vertex) and column offset DV
template <int C, int LD, int I>
__device__ __forceinline__ void bt_pair_term(const float* sp, float2 (&btA)[4], float2 (&btB)[4]) {
    constexpr int RV = I / 3 - 1, DV = I % 3 - 1;
    constexpr int VA = (RV + 1) * 3 + DV + 1, VB = RV * 3 + DV + 1;
    constexpr bool useA = RV <= 1 && bt_vwin(C, VA), useB = RV >= 0 && bt_vwin(C, VB);
    if constexpr (useA || useB) {
        const float v = sp[RV * LD + DV];
        if constexpr (useA) bt_apply<C, (useA ? VA : 0)>(v, btA);
        if constexpr (useB) bt_apply<C, (useB ? VB : 0)>(v, btB);
    }
}
template <int C, int LD, int... I>
__device__ __forceinline__ void bt_pair_rows(const float* sp, float2 (&btA)[4], float2 (&btB)[4],
                                             std::integer_sequence<int, I...>) {
    (bt_pair_term<C, LD, I>(sp, btA, btB), ...);
}
// B row of the vertices of rows r (A) and r + 1 (B) over the u^{m-1/2} planes
template <int C, int FW, int I>
__device__ __forceinline__ void b_pair_term(const float2* f0, int fpl, float& accA, float& accB) {
    constexpr int R = I / 5 - 2, DX = I % 5 - 2;
    constexpr int WA = (R + 2) * 5 + DX + 2, WB = R * 5 + DX + 2;
    constexpr bool useA = R <= 2 && (kBx[C][R <= 2 ? WA : 0] != 0 || kBy[C][R <= 2 ? WA : 0] != 0);
    constexpr bool useB = R >= 0 && (kBx[C][R >= 0 ? WB : 0] != 0 || kBy[C][R >= 0 ? WB : 0] != 0);
    if constexpr (useA || useB) {
        constexpr int plane = (DX & 1) + 2 * (R & 1);
        const float2 w = f0[plane * fpl + (R >> 1) * FW + (DX >> 1)];
        if constexpr (useA) {
            addk<kBx[C][useA ? WA : 0]>(accA, w.x);
            addk<kBy[C][useA ? WA : 0]>(accA, w.y);
        }
        if constexpr (useB) {
            addk<kBx[C][useB ? WB : 0]>(accB, w.x);
            addk<kBy[C][useB ? WB : 0]>(accB, w.y);
        }
    }
}
template <int C, int FW, int... I>
__device__ __forceinline__ void b_pair_rows(const float2* f0, int fpl, float& accA, float& accB,
                                            std::integer_sequence<int, I...>) {
    (b_pair_term<C, FW, I>(f0, fpl, accA, accB), ...);
}

// u^{m-1/2} of the cells of row r from their A and B^T rows (written over f)
template <class G, bool INNER>
__device__ __forceinline__ void u_half_row(const float2 (&au)[4], const float2 (&ctr)[4], const float2 (&bt)[4],
                                           float ti0, float ti1, float2 mb, float2* sF, int FPL, int r, int lane,
                                           int i0, int j0, int n) {
    bool unk[4] = {true, true, true, true};
    if constexpr (!INNER) {
        const int ci = i0 - 2 + lane, cj = j0 - 2 + r;
        const bool ci_in = ci > 0 && ci < n, cj_in = cj > 0 && cj < n;
        const bool ci_h = ci >= 0 && ci < n, cj_h = cj >= 0 && cj < n;
        unk[0] = ci_in && cj_in;
        unk[1] = ci_h && cj_in;
        unk[2] = ci_in && cj_h;
        unk[3] = ci_h && cj_h;
    }
    float2* fr = sF + r * G::FW + lane;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float2 fs = fr[s * FPL];
        const float ti = s == 0 ? ti0 : ti1;
        float2 t = f2(fs.x - au[s].x, fs.y - au[s].y);
        if (s > 0) t = __ffma2_rn(mb, bt[s], t);
        const float2 h = __ffma2_rn(f2(ti, ti), t, ctr[s]);
        if constexpr (INNER) fr[s * FPL] = h;
        else fr[s * FPL] = unk[s] ? h : f2(0.f, 0.f);
    }
}

template <class G, int C, bool INNER>
__device__ __forceinline__ void phase1_pair(const RegCoef& q, const float2* sU, int UPL, const float* sP, float2* sF,
                                           int FPL, int TY, int NW, int warp, int lane, int i0, int j0, int n) {
    float2 a[kGroups];
    load_coef<C>(q, a);
    const float ti0 = q.ti[C][0], ti1 = q.ti[C][1];
    const float2 mb = f2(-q.b, -q.b);
    for (int r = 2 * warp; r < TY + 4; r += 2 * NW) {
        const float2* t0 = sU + 2 * (r + 1) * G::UWH + lane + G::UX - 2;
        const float2* t1 = t0 + UPL;
        float2 auA[4], ctrA[4], btA[4], auB[4], ctrB[4], btB[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) auA[s] = ctrA[s] = btA[s] = auB[s] = ctrB[s] = btB[s] = f2(0.f, 0.f);
        a_pair_rows<C, G::UWH>(a, t0, t1, auA, ctrA, auB, ctrB, std::make_integer_sequence<int, 35>{});
        bt_pair_rows<C, G::PW>(sP + (r + 1) * G::PW + lane + G::PX - 2, btA, btB, std::make_integer_sequence<int, 12>{});
        u_half_row<G, INNER>(auA, ctrA, btA, ti0, ti1, mb, sF, FPL, r, lane, i0, j0, n);
        u_half_row<G, INNER>(auB, ctrB, btB, ti0, ti1, mb, sF, FPL, r + 1, lane, i0, j0, n);
    }
}

template <class G, int C>
__device__ __forceinline__ void phase2_pair(const RegCoef& q, const float2* sF, int FPL, float* sG, const float* sS,
                                            float sigma, int TY, int NW, int warp, int lane) {
    const float b = q.b;
    for (int r = 2 * warp; r < TY + 2; r += 2 * NW) {
        if (lane >= G::DN) break;
        const float2* f0 = sF + (r + 1) * G::FW + lane + 1;
        float accA = 0.f, accB = 0.f;
        b_pair_rows<C, G::FW>(f0, FPL, accA, accB, std::make_integer_sequence<int, 35>{});
        const int k = r * G::DW + lane + G::DX - 1;
        sG[k] = sigma * sS[k] * fmaf(b, accA, -sG[k]);
        sG[k + G::DW] = sigma * sS[k + G::DW] * fmaf(b, accB, -sG[k + G::DW]);
    }
}

// the new (u, p) of the cells of row r from their B^T dp rows
template <class G, bool PLO, bool INNER>
__device__ __forceinline__ void uzawa_out_row(const float2 (&bt)[4], float nb1, const float2* sF, int FPL,
                                              const float* sG, const float* sP, int r, int lane, int i0, int j0,
                                              int n, float* __restrict__ u_out, float* __restrict__ p_out) {
    const int ci = i0 + lane, cj = j0 + r;
    if (!INNER && (ci > n || cj > n)) return;
    const float2* hr = sF + (r + 2) * G::FW + lane + 2;
    float2 o[4];
    o[0] = hr[0];
#pragma unroll
    for (int s = 1; s < 4; ++s) o[s] = __ffma2_rn(f2(nb1, nb1), bt[s], hr[s * FPL]);
    if constexpr (INNER) {
#pragma unroll
        for (int s = 0; s < 4; ++s) store_node<PLO>(u_out, n, 2 * ci + (s & 1), 2 * cj + (s >> 1), o[s]);
    } else {
        const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            store_node<PLO>(u_out, n, 2 * ci + (s & 1), 2 * cj + (s >> 1), slot_unknown(cn, s) ? o[s] : f2(0.f, 0.f));
        }
    }
    p_out[vert_at<PLO>(n, ci, cj)] = sP[(r + 3) * G::PW + lane + G::PX] + sG[(r + 1) * G::DW + lane + G::DX];
}

template <class G, bool PLO, int C, bool INNER>
__device__ __forceinline__ void phase3_pair(const RegCoef& q, const float2* sF, int FPL, const float* sG,
                                            const float* sP, int TY, int NW, int warp, int lane, int i0, int j0,
                                            int n, float* __restrict__ u_out, float* __restrict__ p_out) {
    const float nb1 = -q.ti[C][1] * q.b;
    for (int r = 2 * warp; r < TY; r += 2 * NW) {
        if (lane >= G::TX) break;
        float2 btA[4], btB[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) btA[s] = btB[s] = f2(0.f, 0.f);
        bt_pair_rows<C, G::DW>(sG + (r + 1) * G::DW + lane + G::DX, btA, btB, std::make_integer_sequence<int, 12>{});
        uzawa_out_row<G, PLO, INNER>(btA, nb1, sF, FPL, sG, sP, r, lane, i0, j0, n, u_out, p_out);
        uzawa_out_row<G, PLO, INNER>(btB, nb1, sF, FPL, sG, sP, r + 1, lane, i0, j0, n, u_out, p_out);
    }
}

// The three phases of the step on the staged tiles (sU, sP, sF = f, sG = g, sS = Shat^{-1}); writes
// the new state of the CTA's cells to (u_out, p_out).
template <class G, bool PLO, int NW, bool PAIR = false>
__device__ __forceinline__ void reg_phases(int n, int TY, int i0, int j0, const OpCoef<float>& c, const RegCoef& q,
                                           float tau, float sigma, const float2* sU, float2* sF, const float* sP,
                                           float* sG, const float* sS, float* __restrict__ u_out,
                                           float* __restrict__ p_out) {
    constexpr int TX = G::TX;
    const int UPL = G::upl(TY), FPL = G::fpl(TY);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int h = n >> 1;
    const bool fast = (h < i0 - 2 || h >= i0 + TX + 2) && (h < j0 - 2 || h >= j0 + TY + 2);
    const bool inner = fast && i0 >= 4 && j0 >= 4 && i0 + TX + 3 <= n && j0 + TY + 3 <= n;
    const int cls = orient(i0, j0, n);

    const ULat<G> vux{sU, UPL, i0 - G::UX, 2 * (j0 - 3), false};
    const ULat<G> vuy{sU, UPL, i0 - G::UX, 2 * (j0 - 3), true};
    const SVert<float, G::PW> vp{sP, i0 - G::PX, j0 - 3};
    const QuadLat<G> vhx{sF, FPL, i0 - 2, j0 - 2, false};
    const QuadLat<G> vhy{sF, FPL, i0 - 2, j0 - 2, true};

    // ---- u^{m-1/2} on cells (i0 - 2 + lane, j0 - 2 + r), written over f
    if (fast && PAIR) {
        if (inner) {
            if (cls == 0) phase1_pair<G, 0, true>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
            else phase1_pair<G, 1, true>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
        } else {
            if (cls == 0) phase1_pair<G, 0, false>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
            else phase1_pair<G, 1, false>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
        }
    } else if (fast) {
        if (inner) {
            if (cls == 0) phase1_fast<G, 0, true>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
            else phase1_fast<G, 1, true>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
        } else {
            if (cls == 0) phase1_fast<G, 0, false>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
            else phase1_fast<G, 1, false>(q, sU, UPL, sP, sF, FPL, TY, NW, warp, lane, i0, j0, n);
        }
    } else {
        for (int r = warp; r < TY + 4; r += NW) {
            const int ci = i0 - 2 + lane, cj = j0 - 2 + r;
            float2 hv[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) hv[s] = f2(0.f, 0.f);
            float2* fr = sF + r * G::FW + lane;
            if (ci >= 0 && cj >= 0 && ci <= n && cj <= n) {
                Acc<float> a;
                cell_apply_auto<true, true, false, true, false>(ci, cj, n, c, vux, vuy, vp, a);
                const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    if (!slot_unknown(cn, s)) continue;
                    const float2 fs = fr[s * FPL];
                    const float w = tau * a.idg[s];
                    hv[s] = f2(vux.at(ci, cj, s & 1, s >> 1) + w * (fs.x - a.au[0][s] - a.bt[0][s]),
                               vuy.at(ci, cj, s & 1, s >> 1) + w * (fs.y - a.au[1][s] - a.bt[1][s]));
                }
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) fr[s * FPL] = hv[s];
        }
    }
    __syncthreads();

    // ---- dp on vertices (i0 - 1 + lane, j0 - 1 + r), written over g
    if (fast && PAIR) {
        if (cls == 0) phase2_pair<G, 0>(q, sF, FPL, sG, sS, sigma, TY, NW, warp, lane);
        else phase2_pair<G, 1>(q, sF, FPL, sG, sS, sigma, TY, NW, warp, lane);
    } else if (fast) {
        if (cls == 0) phase2_fast<G, 0>(q, sF, FPL, sG, sS, sigma, TY, NW, warp, lane);
        else phase2_fast<G, 1>(q, sF, FPL, sG, sS, sigma, TY, NW, warp, lane);
    } else {
        for (int r = warp; r < TY + 2; r += NW) {
            if (lane >= G::DN) break;
            const int vi = i0 - 1 + lane, vj = j0 - 1 + r;
            const int k = r * G::DW + lane + G::DX - 1;
            float d = 0.f;
            if (vi >= 0 && vj >= 0 && vi <= n && vj <= n) {
                Acc<float> a;
                cell_apply_auto<false, false, true, false, false>(vi, vj, n, c, vhx, vhy, vp, a);
                d = sigma * sS[k] * (a.bu - sG[k]);
            }
            sG[k] = d;
        }
    }
    __syncthreads();

    // ---- new (u, p) on the owned cells (i0 + lane, j0 + r)
    if (fast && PAIR) {
        if (inner) {
            if (cls == 0) phase3_pair<G, PLO, 0, true>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
            else phase3_pair<G, PLO, 1, true>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
        } else {
            if (cls == 0) phase3_pair<G, PLO, 0, false>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
            else phase3_pair<G, PLO, 1, false>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
        }
    } else if (fast) {
        if (inner) {
            if (cls == 0) phase3_fast<G, PLO, 0, true>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
            else phase3_fast<G, PLO, 1, true>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
        } else {
            if (cls == 0) phase3_fast<G, PLO, 0, false>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
            else phase3_fast<G, PLO, 1, false>(q, sF, FPL, sG, sP, TY, NW, warp, lane, i0, j0, n, u_out, p_out);
        }
    } else {
        const SVert<float, G::DW> vd{sG, i0 - G::DX, j0 - 1};
        for (int r = warp; r < TY; r += NW) {
            if (lane >= TX) break;
            const int ci = i0 + lane, cj = j0 + r;
            if (ci > n || cj > n) continue;
            Acc<float> a;
            cell_apply_auto<false, true, false, true, false>(ci, cj, n, c, vhx, vhy, vd, a);
            const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!slot_exists(cn, s)) continue;
                float2 o = f2(0.f, 0.f);
                if (slot_unknown(cn, s)) {
                    const float w = tau * a.idg[s];
                    o = f2(vhx.at(ci, cj, s & 1, s >> 1) - w * a.bt[0][s], vhy.at(ci, cj, s & 1, s >> 1) - w * a.bt[1][s]);
                }
                store_node<PLO>(u_out, n, 2 * ci + (s & 1), 2 * cj + (s >> 1), o);
            }
            p_out[vert_at<PLO>(n, ci, cj)] = sP[(r + 3) * G::PW + lane + G::PX] + sG[(r + 1) * G::DW + lane + G::DX];
        }
    }
}

template <int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB)
    k_uzawa_reg(int n, int TY, TileOrder ord, const __grid_constant__ OpCoef<float> c, const __grid_constant__ RegCoef q,
                float tau, float sigma, const float* __restrict__ u, const float* __restrict__ p,
                const float* __restrict__ f, const float* __restrict__ g, const float* __restrict__ sinv,
                float* __restrict__ u_out, float* __restrict__ p_out) {
    pdl_wait();
    using G = RegTile;
    constexpr int TX = G::TX;
    const int UPL = G::upl(TY), FPL = G::fpl(TY), DSZ = G::dsz(TY);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sU = reinterpret_cast<float2*>(smem_raw);
    float2* sF = sU + 2 * UPL;
    float* sP = reinterpret_cast<float*>(sF + 4 * FPL);
    float* sG = sP + G::PW * (TY + 6);
    float* sS = sG + DSZ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int tc, tr;
    ord.tile(blockIdx.x, tc, tr);
    const int i0 = tc * TX, j0 = tr * TY;
    const int ld = 2 * n + 1, n2 = ld * ld, h = n >> 1;
    const bool fast = (h < i0 - 2 || h >= i0 + TX + 2) && (h < j0 - 2 || h >= j0 + TY + 2);
    const bool inner = fast && i0 >= 4 && j0 >= 4 && i0 + TX + 3 <= n && j0 + TY + 3 <= n;

    // ---- asynchronous staging.  Lane l copies component l >> 4 of lattice point 16 q + (l & 15) of a row:
    // one instruction moves 16 consecutive points with both components (two 64-byte global segments,
    // 32 distinct shared banks).  Interior tiles copy without any test, at fixed offsets from one
    // address per row; the others zero-fill what lies off the domain (u also on its boundary).
    {
        const int cx = lane >> 4, px = lane & 15;
        // u: lattice columns X0 + x, x in [0, 68), rows Y0 + y, y in [0, 2 (TY + 6)); column x goes to plane
        // x & 1, plane column x >> 1
        const int X0 = 2 * (i0 - 3), Y0 = 2 * (j0 - 3);
        float* du = reinterpret_cast<float*>(sU + (px & 1) * UPL + (px >> 1)) + cx;
        const float* gu = u + cx * n2 + X0 + px;
        for (int y = warp; y < 2 * (TY + 6); y += NW) {
            const int Y = Y0 + y;
            float* d = du + 2 * y * G::UWH;
            if (inner) {
                const float* src = gu + Y * ld;
#pragma unroll
                for (int t = 0; t < 4; ++t) cp4(d + 16 * t, src + 16 * t, true);
                if (px < 4) cp4(d + 64, src + 64, true);
            } else {
#pragma unroll
                for (int t = 0; t < 5; ++t) {
                    if (t == 4 && px >= 4) break;
                    const bool ok = interior2(X0 + px + 16 * t, Y, n);
                    cp4(d + 16 * t, ok ? gu + Y * ld + 16 * t : u, ok);
                }
            }
        }
        // f: the u^{m-1/2} region, lattice columns XF + x, x in [0, 64), rows YF + y; node type
        // (x & 1) + 2 (y & 1), cell (x >> 1, y >> 1)
        const int XF = 2 * (i0 - 2), YF = 2 * (j0 - 2);
        float* dfb = reinterpret_cast<float*>(sF + (px & 1) * FPL + (px >> 1)) + cx;
        const float* gf = f + cx * n2 + XF + px;
        for (int y = warp; y < 2 * (TY + 4); y += NW) {
            const int Y = YF + y;
            float* d = dfb + 2 * ((y & 1) * 2 * FPL + (y >> 1) * G::FW);
            if (inner) {
                const float* src = gf + Y * ld;
#pragma unroll
                for (int t = 0; t < 4; ++t) cp4(d + 16 * t, src + 16 * t, true);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int X = XF + px + 16 * t;
                    const bool ok = X >= 0 && Y >= 0 && X <= 2 * n && Y <= 2 * n;
                    cp4(d + 16 * t, ok ? gf + Y * ld + 16 * t : f, ok);
                }
            }
        }
        // p: vertices (i0 - 3 + x, j0 - 3 + y), x in [0, 34)
        for (int y = warp; y < TY + 6; y += NW) {
            const int J = j0 - 3 + y;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (t == 1 && lane >= 2) break;
                const int x = lane + 32 * t, I = i0 - 3 + x;
                const bool ok = inner || (I >= 0 && J >= 0 && I <= n && J <= n);
                cp4(sP + y * G::PW + x, ok ? p + J * (n + 1) + I : p, ok);
            }
        }
        // g, Shat^{-1}: vertices (i0 - 1 + x, j0 - 1 + y), x in [0, 30)
        for (int y = warp; y < TY + 2; y += NW) {
            if (lane >= G::DW) break;
            const int J = j0 - 1 + y, I = i0 - 1 + lane;
            const bool ok = inner || (I >= 0 && J >= 0 && I <= n && J <= n);
            const int k = ok ? J * (n + 1) + I : 0;
            cp4(sG + y * G::DW + lane, g + k, ok);
            cp4(sS + y * G::DW + lane, sinv + k, ok);
        }
        cp_commit_wait();
    }
    __syncthreads();


    reg_phases<G, false, NW>(n, TY, i0, j0, c, q, tau, sigma, sU, sF, sP, sG, sS, u_out, p_out);
    pdl_trigger();
}

// ---------------------------------------------------------------------------------------------
// The step on planar float32 levels: the five input tiles arrive by tensor-memory-access box copies
// (cp.async.bulk.tensor into the CTA's own shared memory, completion counted on one mbarrier), so
// staging issues no per-thread load instructions; zero fill outside the arrays and the layout's
// zero boundary and padding replace the masking of the asynchronous-copy path.

struct TmaMaps {
    CUtensorMap u;        // velocity, 3-d: (2 pl_pitch floats, pl_rows rows, 2 parity planes)
    CUtensorMap f0, f1;   // right-hand side at even / odd rows, 3-d: (floats, cell rows, parity planes)
    CUtensorMap p, g, s;  // vertex arrays, 2-d: (pl_vpitch floats, N + 1 rows)
};

// Set (never cleared by the kernels) when a CTA gave up waiting for its tiles; read and cleared by
// uzawa_tma_timeouts().
__device__ unsigned g_tma_timeout = 0;

constexpr long long kTmaWaitCycles = 2000000000LL;   // about one second at the GPU's clock

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on phase `parity` of the mbarrier at shared address bar; false after about a second
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kTmaWaitCycles) return false;
    return true;
}
__device__ __forceinline__ void tma_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_3d(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(map), "r"(x), "r"(y) : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(map), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
// the five tiles of the tile at (i0, j0) into L2, for the CTA that will take that tile later
__device__ __forceinline__ void tma_prefetch_tile(int TY, int i0, int j0, const TmaMaps& maps) {
    using G = TmaTile;
    tma_prefetch_3d(&maps.u, 2 * (i0 - G::UX), 2 * (j0 - 3), 0);
    tma_prefetch_3d(&maps.f0, 2 * (i0 - 2), j0 - 2, 0);
    tma_prefetch_3d(&maps.f1, 2 * (i0 - 2), j0 - 2, 0);
    tma_prefetch_2d(&maps.p, i0 - G::PX, j0 - 3);
    tma_prefetch_2d(&maps.g, i0 - G::DX, j0 - 1);
    tma_prefetch_2d(&maps.s, i0 - G::DX, j0 - 1);
}

// ---- the coarse-grid correction x += P x_c (Sec. 3, the canonical embedding) on the staged u and
// p tiles of the first post-smoothing step: every fine lattice point of the u tile and every fine
// vertex of the p tile gets the coarse P2 / P1 function of the coarse square that owns it, added in
// shared memory, so the corrected state is never written to global memory and read back.

// the two triangles of a coarse square of orientation o (the split of tri_mask), vertices in coarse
// lattice units (0 or 2)
struct EmbedTri {
    int x[3], y[3];
};
__host__ __device__ constexpr EmbedTri embed_tri(int o, int t) {
    return o == 0 ? (t == 0 ? EmbedTri{{0, 2, 2}, {0, 0, 2}} : EmbedTri{{0, 2, 0}, {0, 2, 2}})
                  : (t == 0 ? EmbedTri{{0, 2, 0}, {0, 0, 2}} : EmbedTri{{2, 2, 0}, {0, 2, 2}});
}
// Value at the fine lattice point (fa / 2, fb / 2), fa, fb in [0, 4), of the coarse P2 basis
// function of local node L (lattice offset (L % 3, L / 3)): in the triangle that holds the point,
// with barycentric coordinates l, l_i (2 l_i - 1) at vertex i and 4 l_j l_k at the midpoint of the
// edge (j, k); zero where L is no node of that triangle.  Evaluated at compile time.
__host__ __device__ constexpr double embed_weight(int o, int L, int fa, int fb) {
    const double px = 0.5 * fa, py = 0.5 * fb;
    const int lx = L % 3, ly = L / 3;
    for (int t = 0; t < 2; ++t) {
        const EmbedTri T = embed_tri(o, t);
        const double twoA = (T.x[1] - T.x[0]) * (T.y[2] - T.y[0]) - (T.x[2] - T.x[0]) * (T.y[1] - T.y[0]);
        double l[3] = {0.0, 0.0, 0.0};
        bool inside = true;
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3, k = (i + 2) % 3;
            l[i] = ((T.x[j] - px) * (T.y[k] - py) - (T.x[k] - px) * (T.y[j] - py)) / twoA;
            if (l[i] < 0.0) inside = false;
        }
        if (!inside) continue;
        for (int i = 0; i < 3; ++i)
            if (T.x[i] == lx && T.y[i] == ly) return l[i] * (2.0 * l[i] - 1.0);
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3, k = (i + 2) % 3;
            if (T.x[j] + T.x[k] == 2 * lx && T.y[j] + T.y[k] == 2 * ly) return 4.0 * l[j] * l[k];
        }
        return 0.0;
    }
    return 0.0;
}
__host__ __device__ constexpr bool embed_partition_of_unity() {
    for (int o = 0; o < 2; ++o)
        for (int f = 0; f < 16; ++f) {
            double s = 0.0;
            for (int L = 0; L < 9; ++L) s += embed_weight(o, L, f % 4, f / 4);
            if (s != 1.0) return false;
        }
    return true;
}
static_assert(embed_partition_of_unity(), "the coarse basis functions sum to one at every fine point");
static_assert(embed_weight(0, 0, 1, 0) == 0.375 && embed_weight(0, 1, 1, 0) == 0.75 && embed_weight(0, 2, 1, 0) == -0.125,
              "on a coarse edge the embedding is the quadratic through its three nodes");
static_assert(embed_weight(1, 4, 2, 2) == 1.0 && embed_weight(0, 3, 2, 2) == 0.0, "a coarse node keeps its value");

template <int O, int FA, int FB, int L>
__device__ __forceinline__ void embed_term(const float2 (&z)[9], float2& acc) {
    constexpr float w = (float)embed_weight(O, L, FA, FB);
    if constexpr (w == 1.0f) acc = f2(acc.x + z[L].x, acc.y + z[L].y);
    else if constexpr (w != 0.0f) acc = __ffma2_rn(f2(w, w), z[L], acc);
}
// fine point P = FB * 4 + FA of a coarse square added to its u-tile entry (plane FA & 1, row FB,
// pair FA / 2 from the square's corner at offset `base` of plane 0) if bit P of `mask` is set
template <class G, int O, int P, int... L>
__device__ __forceinline__ void embed_point(const float2 (&z)[9], float2* sU, int base, int UPL, unsigned mask,
                                            std::integer_sequence<int, L...>) {
    constexpr int FA = P % 4, FB = P / 4;
    if (!((mask >> P) & 1u)) return;
    float2* d = sU + base + (FA & 1) * UPL + FB * G::UWH + (FA >> 1);
    float2 acc = *d;
    (embed_term<O, FA, FB, L>(z, acc), ...);
    *d = acc;
}
template <class G, int O, int... P>
__device__ __forceinline__ void embed_square(const float2 (&z)[9], float2* sU, int base, int UPL, unsigned mask,
                                             std::integer_sequence<int, P...>) {
    (embed_point<G, O, P>(z, sU, base, UPL, mask, std::make_integer_sequence<int, 9>{}), ...);
}
// the same for a square whose 16 points all lie in the tile and inside the level: the 16 tile
// entries are read first, corrected, then written (no per-point tests); b0, b1 = the square's
// corner in the two column-parity planes
template <class G, int P>
__device__ __forceinline__ float2* embed_at(float2* b0, float2* b1) {
    return ((P % 4) & 1 ? b1 : b0) + (P / 4) * G::UWH + ((P % 4) >> 1);
}
template <int O, int P, int... L>
__device__ __forceinline__ void embed_fma(const float2 (&z)[9], float2& v, std::integer_sequence<int, L...>) {
    (embed_term<O, P % 4, P / 4, L>(z, v), ...);
}
template <class G, int O, int P0, int... P>
__device__ __forceinline__ void embed_chunk(const float2 (&z)[9], float2* b0, float2* b1, std::integer_sequence<int, P...>) {
    float2 v[sizeof...(P)];
    ((v[P] = *embed_at<G, P0 + P>(b0, b1)), ...);
    (embed_fma<O, P0 + P>(z, v[P], std::make_integer_sequence<int, 9>{}), ...);
    ((*embed_at<G, P0 + P>(b0, b1) = v[P]), ...);
}
// CH points at a time (16, or 8 where registers are scarce)
template <class G, int O, int CH>
__device__ __forceinline__ void embed_square_full(const float2 (&z)[9], float2* b0, float2* b1) {
    static_assert(CH == 8 || CH == 16, "whole rows of points");
    embed_chunk<G, O, 0>(z, b0, b1, std::make_integer_sequence<int, CH>{});
    if constexpr (CH == 8) embed_chunk<G, O, 8>(z, b0, b1, std::make_integer_sequence<int, 8>{});
}

// One coarse square's share of the correction: its nine P2 values and the P1 values at its four
// corners (those of the level), loaded before the tiles arrive.
struct EmbedJob {
    float2 z[9];
    float p00, p10, p01, p11;
    int I, J;   // I < 0: no work
};

// The coarse squares [i0 / 2 - 2, i0 / 2 + 16) x [J0, J1] of the CTA at (i0, j0) own every fine
// lattice point of its u tile (pairs from cell i0 - UX, rows from 2 (j0 - 3)) and every fine vertex of
// its p tile (from (i0 - PX, j0 - 3)); job t is square (I0 + t % 18, J0 + t / 18).
template <class G>
struct EmbedGrid {
    static constexpr int NI = G::UWH / 2;
    static_assert(G::UX == 4 && G::PX == 4 && G::UWH % 2 == 0 && G::PW == G::UWH, "tile origin at an even cell");
    int I0, J0, count;
    __device__ __forceinline__ EmbedGrid(int TY, int i0, int j0) {
        I0 = (i0 >> 1) - 2;                   // i0 is even
        J0 = (2 * j0 + 2) / 4 - 2;            // floor((2 j0 - 6) / 4) for j0 >= 0
        count = NI * ((2 * j0 + 2 * TY + 5) / 4 - J0 + 1);
    }
};

// Tile height of the launches that add the correction: at most 18 x 14 coarse squares, so that each
// of the 256 threads has one square at most (a second square for a few threads left the other
// warps waiting on them).
constexpr int kEmbedMaxRows = 20;
constexpr int embed_max_squares(int ty) {   // over tile origins j0 of either parity
    const int even = (2 * ty + 5) / 4 + 3, odd = (2 * ty + 7) / 4 + 2;
    return EmbedGrid<TmaTile>::NI * (even > odd ? even : odd);
}
static_assert(embed_max_squares(kEmbedMaxRows) <= 256, "one coarse square per thread");

// coarse iterate (uc, pc) of level nc, planar when pcp
__device__ __forceinline__ void embed_load(EmbedJob& jb, int t, const EmbedGrid<TmaTile>& eg, int nc,
                                           const float* __restrict__ uc, const float* __restrict__ pc, bool pcp) {
    constexpr int NI = EmbedGrid<TmaTile>::NI;
    const int I = eg.I0 + t % NI, J = eg.J0 + t / NI;
    jb.I = -1;
    if (t >= eg.count || I < 0 || J < 0 || I > nc || J > nc) return;
    jb.I = I;
    jb.J = J;
    const int ldc = 2 * nc + 1, vld = pcp ? pl_vpitch(nc) : nc + 1;
    if (I < nc && J < nc) {
        if (pcp) {   // pair I (+1) of rows 2J .. 2J + 2 of the two column-parity planes
            const float2* r0 = reinterpret_cast<const float2*>(uc + pl_u(nc, 2 * I, 2 * J));
            const int rp = pl_pitch(nc), pp = pl_rows(nc) * pl_pitch(nc);
#pragma unroll
            for (int m = 0; m < 9; ++m) jb.z[m] = __ldg(r0 + (m % 3 & 1) * pp + (m / 3) * rp + (m % 3 >> 1));
        } else {
            const float* r0 = uc + (2 * J) * ldc + 2 * I;
#pragma unroll
            for (int m = 0; m < 9; ++m) {
                const int k = (m / 3) * ldc + m % 3;
                jb.z[m] = f2(__ldg(r0 + k), __ldg(r0 + ldc * ldc + k));
            }
        }
    }
    jb.p00 = __ldg(pc + J * vld + I);
    jb.p10 = I < nc ? __ldg(pc + J * vld + I + 1) : 0.f;
    jb.p01 = J < nc ? __ldg(pc + (J + 1) * vld + I) : 0.f;
    jb.p11 = I < nc && J < nc ? __ldg(pc + (J + 1) * vld + I + 1) : 0.f;
}

// the job's fine points added to the tiles: the lattice points strictly inside the level and the
// tile's rows, and the vertices of the level inside the p tile
template <class G, int CH>
__device__ __forceinline__ void embed_apply(const EmbedJob& jb, int n, int TY, int i0, int j0, float2* sU, float* sP) {
    if (jb.I < 0) return;
    const int nc = n >> 1, I = jb.I, J = jb.J, UPL = G::upl(TY);
    const int pxlo = i0 - G::PX, pylo = j0 - 3;
    // rows [2J, 2J + 2) of vertices (and so [4J, 4J + 4) of lattice points) inside the tiles, and the
    // square strictly inside the level: every point of it is corrected
    if (I > 0 && J > 0 && I < nc && J < nc && 2 * J >= pylo && 2 * J + 2 <= pylo + TY + 6) {
        const int base = (4 * J - 2 * pylo) * G::UWH + ((4 * I - 2 * (i0 - G::UX)) >> 1);
        const int o = orient(I, J, nc);
        if (o == 0) embed_square_full<G, 0, CH>(jb.z, sU + base, sU + base + UPL);
        else embed_square_full<G, 1, CH>(jb.z, sU + base, sU + base + UPL);
        float* q = sP + (2 * J - pylo) * G::PW + (2 * I - pxlo);
        q[0] += jb.p00;
        q[1] += 0.5f * (jb.p00 + jb.p10);
        q[G::PW] += 0.5f * (jb.p00 + jb.p01);
        q[G::PW + 1] += 0.5f * (o == 0 ? jb.p00 + jb.p11 : jb.p10 + jb.p01);
        return;
    }
    if (I < nc && J < nc) {
        const int xlo = 2 * (i0 - G::UX), ylo = 2 * (j0 - 3), yhi = ylo + 2 * (TY + 6);
        unsigned cols = 0u, mask = 0u;
#pragma unroll
        for (int fa = 0; fa < 4; ++fa) {   // the tile holds every column of its squares
            const int X = 4 * I + fa;
            if (X > 0 && X < 2 * n) cols |= 1u << fa;
        }
#pragma unroll
        for (int fb = 0; fb < 4; ++fb) {
            const int Y = 4 * J + fb;
            if (Y >= ylo && Y < yhi && Y > 0 && Y < 2 * n) mask |= cols << (4 * fb);
        }
        const int base = (4 * J - ylo) * G::UWH + ((4 * I - xlo) >> 1);
        constexpr auto P16 = std::make_integer_sequence<int, 16>{};
        if (orient(I, J, nc) == 0) embed_square<G, 0>(jb.z, sU, base, UPL, mask, P16);
        else embed_square<G, 1>(jb.z, sU, base, UPL, mask, P16);
    }
    // P1: injection at the coarse vertex, averages halfway along the coarse edges from it
    auto addp = [&](int x, int y, float v) {
        if (x < pxlo || x >= pxlo + G::PW || y < pylo || y >= pylo + TY + 6 || x > n || y > n) return;
        sP[(y - pylo) * G::PW + (x - pxlo)] += v;
    };
    addp(2 * I, 2 * J, jb.p00);
    if (I < nc) addp(2 * I + 1, 2 * J, 0.5f * (jb.p00 + jb.p10));
    if (J < nc) addp(2 * I, 2 * J + 1, 0.5f * (jb.p00 + jb.p01));
    if (I < nc && J < nc)
        addp(2 * I + 1, 2 * J + 1, 0.5f * (orient(I, J, nc) == 0 ? jb.p00 + jb.p11 : jb.p10 + jb.p01));
}

// pf > 0: also prefetch into L2 the tiles of tile blockIdx.x + pf (about one wave of resident CTAs
// ahead), so that the CTA that takes it finds its tiles in L2
template <int NW, int MINB, bool PAIR = false>
__global__ void __launch_bounds__(32 * NW, MINB)
    k_uzawa_tma(int n, int TY, TileOrder ord, const __grid_constant__ OpCoef<float> c, const __grid_constant__ RegCoef q,
                float tau, float sigma, const __grid_constant__ TmaMaps maps, float* __restrict__ u_out,
                float* __restrict__ p_out, int pf, const float* __restrict__ uc, const float* __restrict__ pc, int pcp) {
    using G = TmaTile;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float2* sU = reinterpret_cast<float2*>(base + 128);
    float2* sF = reinterpret_cast<float2*>(base + G::off_f(TY));
    float* sP = reinterpret_cast<float*>(base + G::off_p(TY));
    float* sG = reinterpret_cast<float*>(base + G::off_g(TY));
    float* sS = reinterpret_cast<float*>(base + G::off_s(TY));
    const unsigned bar = (unsigned)__cvta_generic_to_shared(base);
    int tc, tr;
    ord.tile(blockIdx.x, tc, tr);
    const int i0 = tc * G::TX, j0 = tr * TY;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();   // the inputs are the previous kernel's outputs
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(G::tx_bytes(TY)) : "memory");
        const unsigned du = (unsigned)__cvta_generic_to_shared(sU), df = (unsigned)__cvta_generic_to_shared(sF);
        tma_3d(du, &maps.u, 2 * (i0 - G::UX), 2 * (j0 - 3), 0, bar);
        tma_3d(df, &maps.f0, 2 * (i0 - 2), j0 - 2, 0, bar);
        tma_3d(df + 8 * 2 * G::fpl(TY), &maps.f1, 2 * (i0 - 2), j0 - 2, 0, bar);
        tma_2d((unsigned)__cvta_generic_to_shared(sP), &maps.p, i0 - G::PX, j0 - 3, bar);
        tma_2d((unsigned)__cvta_generic_to_shared(sG), &maps.g, i0 - G::DX, j0 - 1, bar);
        tma_2d((unsigned)__cvta_generic_to_shared(sS), &maps.s, i0 - G::DX, j0 - 1, bar);
        const int ahead = (int)blockIdx.x + pf;
        if (pf > 0 && ahead < (int)gridDim.x) {
            int ac, ar;
            ord.tile(ahead, ac, ar);
            tma_prefetch_tile(TY, ac * G::TX, ar * TY, maps);
        }
    }
    // uc, pc given: the step starts from x + P x_c; each thread loads the coarse values of its
    // square while the tiles are in flight
    const EmbedGrid<G> eg(TY, i0, j0);
    EmbedJob jb;
    if (uc) embed_load(jb, threadIdx.x, eg, n >> 1, uc, pc, pcp != 0);
    const bool ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(&g_tma_timeout, 1u);
            mbar_wait_bounded(bar, 0);   // once more, for copies still in flight into this CTA's memory
        }
        return;
    }
    if (uc) {
        constexpr int CH = MINB >= 4 ? 8 : 16;   // points corrected at a time (registers)
        embed_apply<G, CH>(jb, n, TY, i0, j0, sU, sP);
        for (int t = threadIdx.x + 32 * NW; t < eg.count; t += 32 * NW) {   // tiles above kEmbedMaxRows only
            embed_load(jb, t, eg, n >> 1, uc, pc, pcp != 0);
            embed_apply<G, CH>(jb, n, TY, i0, j0, sU, sP);
        }
        __syncthreads();
    }
    reg_phases<G, true, NW, PAIR>(n, TY, i0, j0, c, q, tau, sigma, sU, sF, sP, sG, sS, u_out, p_out);
    pdl_trigger();
}

// ---------------------------------------------------------------------------------------------
// Residual and restriction of a planar level in one kernel (Sec. 3: the coarse right-hand side is
// the transposed canonical embedding of the fine defect).  A CTA stages the tiles of k_uzawa_tma
// (the g tile one row lower, no Shat^{-1}), forms the defect r = F - A x on fine cells and vertices
// [i0 - 2, i0 + TX) x [j0 - 2, j0 + ty) in shared memory (r_u over f, r_p over g), and restricts it
// to its own coarse cells [i0 / 2, i0 / 2 + TX / 2) x [j0 / 2, j0 / 2 + ty / 2): every fine point that
// a coarse basis function of those cells reaches lies in that region.  The fine defect never goes to
// global memory.  The coarse iterate of those cells is set to zero (the coarse correction starts
// from 0).

// The canonical embedding weights of the restriction, [orientation][coarse local node][fb][fa]
struct RestrictWeights {
    float w[2][9][4][4];
};

// B row of a vertex over the u tile (two column-parity planes, as a_term reads them)
template <int C, int UWH, int W>
__device__ __forceinline__ void bu_term(const float2* t0, const float2* t1, float& acc) {
    if constexpr (kBx[C][W] != 0 || kBy[C][W] != 0) {
        constexpr int dx = W % 5 - 2, dy = W / 5 - 2;
        const float2 w = ((dx & 1) ? t1 : t0)[dy * UWH + (dx >> 1)];
        addk<kBx[C][W]>(acc, w.x);
        addk<kBy[C][W]>(acc, w.y);
    }
}
template <int C, int UWH, int... W>
__device__ __forceinline__ float bu_row(const float2* t0, const float2* t1, std::integer_sequence<int, W...>) {
    float acc = 0.f;
    (bu_term<C, UWH, W>(t0, t1, acc), ...);
    return acc;
}

// the defect on cells and vertices (i0 - 2 + lane, j0 - 2 + r), r < TY + 2, fast path (class C)
template <class G, int C>
__device__ __forceinline__ void defect_fast(const RegCoef& q, const float2* sU, int UPL, const float* sP, float2* sF,
                                           int FPL, float* sG, int TY, int NW, int warp, int lane, int i0, int j0,
                                           int n) {
    float2 a[kGroups];
    load_coef<C>(q, a);
    const float2 mb = f2(-q.b, -q.b);
    const float hb = q.b;
    for (int r = warp; r < TY + 2; r += NW) {
        const float2* t0 = sU + 2 * (r + 1) * G::UWH + lane + G::UX - 2;
        const float2* t1 = t0 + UPL;
        float2 au[4], ctr[4], bt[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) au[s] = ctr[s] = bt[s] = f2(0.f, 0.f);
        a_rows<C, G::UWH>(a, t0, t1, au, ctr, std::make_integer_sequence<int, 25>{});
        bt_rows<C, G::PW>(sP + (r + 1) * G::PW + lane + G::PX - 2, bt, std::make_integer_sequence<int, 9>{});
        const float bu = hb * bu_row<C, G::UWH>(t0, t1, std::make_integer_sequence<int, 25>{});
        const int ci = i0 - 2 + lane, cj = j0 - 2 + r;
        const bool ci_in = ci > 0 && ci < n, cj_in = cj > 0 && cj < n;
        const bool ci_h = ci >= 0 && ci < n, cj_h = cj >= 0 && cj < n;
        const bool unk[4] = {ci_in && cj_in, ci_h && cj_in, ci_in && cj_h, ci_h && cj_h};
        float2* fr = sF + r * G::FW + lane;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float2 fs = fr[s * FPL];
            float2 t = f2(fs.x - au[s].x, fs.y - au[s].y);
            if (s > 0) t = __ffma2_rn(mb, bt[s], t);
            fr[s * FPL] = unk[s] ? t : f2(0.f, 0.f);
        }
        if (lane < G::DN) {
            const int k = r * G::DW + lane + G::DX - 2;
            const bool live = ci >= 0 && cj >= 0 && ci <= n && cj <= n;
            sG[k] = live ? sG[k] - bu : 0.f;
        }
    }
}

// coarse cell (I, J) of level nc: the restricted defect at its owned nodes and vertex, from the
// fine defect tiles (r_u over the node-type planes of sF, origin cell (xc0, yc0); r_p in sG, origin
// vertex (xv0, yv0), DW per row)
template <class G, int SQ>
__device__ __forceinline__ void restrict_sq(const RestrictWeights& wt, int I, int J, int nc, const float2* sF, int FPL,
                                            int xc0, int yc0, float2 (&acc)[4]) {
    const int SI = I - (SQ & 1), SJ = J - (SQ >> 1);
    if (SI < 0 || SJ < 0 || SI >= nc || SJ >= nc) return;
    const int o = orient(SI, SJ, nc);
    float2 v[4][4];
#pragma unroll
    for (int fb = 0; fb < 4; ++fb)
#pragma unroll
        for (int fa = 0; fa < 4; ++fa)
            v[fb][fa] = sF[((fa & 1) + 2 * (fb & 1)) * FPL + (2 * SJ + (fb >> 1) - yc0) * G::FW + 2 * SI + (fa >> 1) - xc0];
#pragma unroll
    for (int R = 0; R < sq_nrows(SQ); ++R) {
        const int L = sq_row(SQ, R), s = sq_slot(SQ, R);
#pragma unroll
        for (int fb = 0; fb < 4; ++fb)
#pragma unroll
            for (int fa = 0; fa < 4; ++fa) {
                const float w = wt.w[o][L][fb][fa];
                acc[s] = __ffma2_rn(f2(w, w), v[fb][fa], acc[s]);
            }
    }
}

// The defect on fine cells and vertices [i0 - 2, i0 + TX) x [j0 - 2, j0 + TY) of the staged tiles
// (r_u over sF, r_p over sG, whose tile starts at vertex row j0 - 2) and its restriction to the
// coarse cells [i0 / 2, i0 / 2 + TX / 2) x [j0 / 2, j0 / 2 + TY / 2) of level n / 2 (planar: PC), with
// the coarse iterate of those cells set to zero.  All threads of the CTA take part.
template <class G, int NW, bool PC>
__device__ __forceinline__ void defect_restrict(int n, int TY, int i0, int j0, const OpCoef<float>& c, const RegCoef& q,
                                                const RestrictWeights& wt, const float2* sU, float2* sF,
                                                const float* sP, float* sG, float* __restrict__ fc,
                                                float* __restrict__ gc, float* __restrict__ uc,
                                                float* __restrict__ pc) {
    constexpr int TX = G::TX;
    const int UPL = G::upl(TY), FPL = G::fpl(TY);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // ---- the fine defect on cells and vertices [i0 - 2, i0 + TX) x [j0 - 2, j0 + TY)
    const int h = n >> 1;
    const bool fast = (h < i0 - 2 || h >= i0 + TX) && (h < j0 - 2 || h >= j0 + TY);
    if (fast) {
        if (orient(i0, j0, n) == 0) defect_fast<G, 0>(q, sU, UPL, sP, sF, FPL, sG, TY, NW, warp, lane, i0, j0, n);
        else defect_fast<G, 1>(q, sU, UPL, sP, sF, FPL, sG, TY, NW, warp, lane, i0, j0, n);
    } else {
        const ULat<G> vux{sU, UPL, i0 - G::UX, 2 * (j0 - 3), false};
        const ULat<G> vuy{sU, UPL, i0 - G::UX, 2 * (j0 - 3), true};
        const SVert<float, G::PW> vp{sP, i0 - G::PX, j0 - 3};
        for (int r = warp; r < TY + 2; r += NW) {
            const int ci = i0 - 2 + lane, cj = j0 - 2 + r;
            const bool live = ci >= 0 && cj >= 0 && ci <= n && cj <= n;
            float2 rv[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) rv[s] = f2(0.f, 0.f);
            float rpv = 0.f;
            float2* fr = sF + r * G::FW + lane;
            const int k = r * G::DW + lane + G::DX - 2;
            if (live) {
                Acc<float> a;
                cell_apply_auto<true, true, true, false, false>(ci, cj, n, c, vux, vuy, vp, a);
                const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    if (!slot_unknown(cn, s)) continue;
                    const float2 fs = fr[s * FPL];
                    rv[s] = f2(fs.x - a.au[0][s] - a.bt[0][s], fs.y - a.au[1][s] - a.bt[1][s]);
                }
                if (lane < G::DN) rpv = sG[k] - a.bu;
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) fr[s * FPL] = rv[s];
            if (lane < G::DN) sG[k] = rpv;
        }
    }
    __syncthreads();
    // ---- restriction to the coarse cells (I, J) of this tile
    const int nc = n >> 1;
    for (int t = threadIdx.x; t < (TX / 2) * (TY / 2); t += 32 * NW) {
        const int I = i0 / 2 + t % (TX / 2), J = j0 / 2 + t / (TX / 2);
        if (I > nc || J > nc) continue;
        float2 acc[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[s] = f2(0.f, 0.f);
        restrict_sq<G, 0>(wt, I, J, nc, sF, FPL, i0 - 2, j0 - 2, acc);
        restrict_sq<G, 1>(wt, I, J, nc, sF, FPL, i0 - 2, j0 - 2, acc);
        restrict_sq<G, 2>(wt, I, J, nc, sF, FPL, i0 - 2, j0 - 2, acc);
        restrict_sq<G, 3>(wt, I, J, nc, sF, FPL, i0 - 2, j0 - 2, acc);
        const CellNodes cn = cell_nodes(I, J, nc);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            const int X = 2 * I + (s & 1), Y = 2 * J + (s >> 1);
            const float2 v = slot_unknown(cn, s) ? acc[s] : f2(0.f, 0.f);
            if constexpr (PC) {
                const int o = pl_u(nc, X, Y);
                *reinterpret_cast<float2*>(fc + o) = v;
                *reinterpret_cast<float2*>(uc + o) = f2(0.f, 0.f);
            } else {
                const int ld = 2 * nc + 1, o = Y * ld + X;
                fc[o] = v.x;
                fc[ld * ld + o] = v.y;
                uc[o] = 0.f;
                uc[ld * ld + o] = 0.f;
            }
        }
        // P1: the fine vertex (2I, 2J), and halves of the fine vertices halfway along the coarse
        // edges through it (horizontal, vertical, and the diagonal of each square whose cut passes
        // through it)
        const int nf = n, x = 2 * I, y = 2 * J;
        auto R = [&](int xx, int yy) { return sG[(yy - (j0 - 2)) * G::DW + xx - (i0 - G::DX)]; };
        const float sv = R(x, y);
        float half = 0.f;
        if (x > 0) half += R(x - 1, y);
        if (x < nf) half += R(x + 1, y);
        if (y > 0) half += R(x, y - 1);
        if (y < nf) half += R(x, y + 1);
        if (x < nf && y < nf && orient(I, J, nc) == 0) half += R(x + 1, y + 1);
        if (x > 0 && y > 0 && orient(I - 1, J - 1, nc) == 0) half += R(x - 1, y - 1);
        if (x < nf && y > 0 && orient(I, J - 1, nc) == 1) half += R(x + 1, y - 1);
        if (x > 0 && y < nf && orient(I - 1, J, nc) == 1) half += R(x - 1, y + 1);
        const int vi = PC ? J * pl_vpitch(nc) + I : J * (nc + 1) + I;
        gc[vi] = fmaf(0.5f, half, sv);
        pc[vi] = 0.f;
    }
}

template <int NW, int MINB, bool PC>
__global__ void __launch_bounds__(32 * NW, MINB)
    k_restrict_tma(int n, int TY, TileOrder ord, const __grid_constant__ OpCoef<float> c,
                   const __grid_constant__ RegCoef q, const __grid_constant__ RestrictWeights wt,
                   const __grid_constant__ TmaMaps maps, float* __restrict__ fc, float* __restrict__ gc,
                   float* __restrict__ uc, float* __restrict__ pc) {
    using G = TmaTile;
    constexpr int TX = G::TX;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float2* sU = reinterpret_cast<float2*>(base + 128);
    float2* sF = reinterpret_cast<float2*>(base + G::off_f(TY));
    float* sP = reinterpret_cast<float*>(base + G::off_p(TY));
    float* sG = reinterpret_cast<float*>(base + G::off_g(TY));
    const unsigned bar = (unsigned)__cvta_generic_to_shared(base);
    const int FPL = G::fpl(TY);
    int tc, tr;
    ord.tile(blockIdx.x, tc, tr);
    const int i0 = tc * TX, j0 = tr * TY;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();
    if (threadIdx.x == 0) {
        const unsigned bytes = G::tx_bytes(TY) - 4u * (unsigned)G::dsz(TY);   // no Shat^{-1} tile
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        const unsigned du = (unsigned)__cvta_generic_to_shared(sU), df = (unsigned)__cvta_generic_to_shared(sF);
        tma_3d(du, &maps.u, 2 * (i0 - G::UX), 2 * (j0 - 3), 0, bar);
        tma_3d(df, &maps.f0, 2 * (i0 - 2), j0 - 2, 0, bar);
        tma_3d(df + 8 * 2 * FPL, &maps.f1, 2 * (i0 - 2), j0 - 2, 0, bar);
        tma_2d((unsigned)__cvta_generic_to_shared(sP), &maps.p, i0 - G::PX, j0 - 3, bar);
        tma_2d((unsigned)__cvta_generic_to_shared(sG), &maps.g, i0 - G::DX, j0 - 2, bar);
    }
    const bool ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(&g_tma_timeout, 1u);
            mbar_wait_bounded(bar, 0);
        }
        return;
    }
    defect_restrict<G, NW, PC>(n, TY, i0, j0, c, q, wt, sU, sF, sP, sG, fc, gc, uc, pc);
    pdl_trigger();
}

// ---------------------------------------------------------------------------------------------
// The float32 cycle below a small level in ONE cooperative launch.  On levels with N <= 128 a
// multigrid phase is a few thousand cells, and launching one kernel per phase costs far more than
// the arithmetic (a W-cycle visits level l 2^(k - l) times).  Here every CTA of a cooperative grid
// (all resident at once) walks the phases of the whole V- or W-cycle from level `top` down to the
// coarsest level of the iteration, doing its share of each phase's tiles and meeting the others at a
// grid barrier between phases (a counter in global memory, bounded waits).  A phase is: one Uzawa
// step (the register tile of k_uzawa_tma on tiles staged by plain loads from the compact layout),
// defect + restriction (defect_restrict), prolongation + correction, or the exact coarsest solve.
// Values written in one phase are read in the next through L2 (__ldcg), never through the read-only
// or L1 caches.

constexpr int kSmallTop = 6;              // highest level the cooperative cycle takes (N = 128)
constexpr int kSmallTY = 12;              // tile height (even: whole coarse cells per tile)
constexpr int kSmallNW = 8;               // warps per CTA
constexpr int kSmallMaxNb = 2212;         // largest bordered coarse system (coarsest level 3)

struct SmallLevelArgs {
    float *u, *p, *f, *g, *tu, *tp;
    const float* sinv;
};
struct SmallCycleArgs {
    SmallLevelArgs L[kSmallTop + 1];      // index = level (N = 2^(level + 1)), compact float32 layout
    RegCoef q[kSmallTop + 1];
    const OpCoef<float>* coef;            // device copies of the levels' operators, index = level
    RestrictWeights wt;
    const double* inv0;                   // level-0 bordered inverse (27 x 27), coarsest level 0
    const double* cinv;                   // coarsest level c > 0: its bordered inverse, cnb x cnb
    int cnb;
    unsigned* bar;                        // barrier counter, zero at launch
    float tau, sigma;
    int nu_pre, nu_post, gamma, top, clev;
};

// Grid barrier number k (k = 1, 2, ...): every CTA adds one to the counter and waits until it
// reaches k x gridDim.x (the counter only grows during a launch).  The wait gives up after about a
// second (g_tma_timeout is set, false is returned).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned k) {
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = k * gridDim.x;
        const long long t0 = clock64();
        // poll with relaxed loads (an acquire load per poll would invalidate the L1 each time); one
        // fence after the wait orders this CTA's later reads after the other CTAs' writes
        while (true) {
            unsigned v;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (clock64() - t0 > kTmaWaitCycles) {
                atomicOr(&g_tma_timeout, 1u);
                ok = false;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    return __syncthreads_and(ok);
}

// Stages the tiles of TmaTile geometry for tile (i0, j0) of a compact float32 level with N = n from
// global memory through L2: u (zero off the interior lattice), f, p, g (vertex rows from gy0) and,
// if sinv is given, Shat^{-1}; zero outside the arrays.
__device__ void stage_compact(int n, int TY, int i0, int j0, int gy0, const float* u, const float* p, const float* f,
                              const float* g, const float* sinv, float2* sU, float2* sF, float* sP, float* sG,
                              float* sS) {
    using G = TmaTile;
    constexpr int B = 4;   // elements per thread and round: their loads are all in flight together
    const int ld = 2 * n + 1, n2 = ld * ld;
    const int nt = blockDim.x;
    // u: two parity planes of 2 (TY + 6) rows of UWH pairs, lattice X = 2 (i0 - UX) + 2 x + plane
    const int un = 2 * 2 * (TY + 6) * G::UWH;
    for (int t0 = threadIdx.x; t0 < un; t0 += B * nt) {
        float2 v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int t = t0 + b * nt;
            const int x = t % G::UWH, y = (t / G::UWH) % (2 * (TY + 6)), pl = t / (G::UWH * 2 * (TY + 6));
            const int X = 2 * (i0 - G::UX) + 2 * x + pl, Y = 2 * (j0 - 3) + y;
            v[b] = (t < un && interior2(X, Y, n)) ? make_float2(__ldcg(u + Y * ld + X), __ldcg(u + n2 + Y * ld + X))
                                                  : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (t0 + b * nt < un) sU[t0 + b * nt] = v[b];
    }
    // f: four node-type planes of TY + 4 cell rows of FW pairs
    const int fn = 4 * (TY + 4) * G::FW;
    for (int t0 = threadIdx.x; t0 < fn; t0 += B * nt) {
        float2 v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int t = t0 + b * nt;
            const int x = t % G::FW, r = (t / G::FW) % (TY + 4), pl = t / (G::FW * (TY + 4));
            const int X = 2 * (i0 - 2 + x) + (pl & 1), Y = 2 * (j0 - 2 + r) + (pl >> 1);
            v[b] = (t < fn && X >= 0 && Y >= 0 && X <= 2 * n && Y <= 2 * n)
                       ? make_float2(__ldcg(f + Y * ld + X), __ldcg(f + n2 + Y * ld + X))
                       : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (t0 + b * nt < fn) sF[t0 + b * nt] = v[b];
    }
    const int pn = (TY + 6) * G::PW, dn = (TY + 2) * G::DW;
    for (int t0 = threadIdx.x; t0 < pn; t0 += B * nt) {
        float v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int t = t0 + b * nt;
            const int I = i0 - G::PX + t % G::PW, J = j0 - 3 + t / G::PW;
            v[b] = (t < pn && I >= 0 && J >= 0 && I <= n && J <= n) ? __ldcg(p + J * (n + 1) + I) : 0.f;
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (t0 + b * nt < pn) sP[t0 + b * nt] = v[b];
    }
    for (int t0 = threadIdx.x; t0 < dn; t0 += B * nt) {
        float vg[B], vs[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int t = t0 + b * nt;
            const int I = i0 - G::DX + t % G::DW, J = gy0 + t / G::DW;
            const bool in = t < dn && I >= 0 && J >= 0 && I <= n && J <= n;
            vg[b] = in ? __ldcg(g + J * (n + 1) + I) : 0.f;
            vs[b] = (in && sinv) ? __ldcg(sinv + J * (n + 1) + I) : 0.f;
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (t0 + b * nt < dn) {
                sG[t0 + b * nt] = vg[b];
                if (sinv) sS[t0 + b * nt] = vs[b];
            }
    }
}

// (u, p) += I (uc, pc) on the fine cells owned by coarse cell (i, j), compact layouts
__device__ void small_prolong_cell(int i, int j, int nc, const RestrictWeights& wt, const float* uc, const float* pc,
                                   float* u, float* p) {
    const int nf = 2 * nc, ldc = 2 * nc + 1, n2c = ldc * ldc, ldf = 2 * nf + 1, n2f = ldf * ldf;
    if (i < nc && j < nc) {
        float zx[9], zy[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int k = (2 * j + m / 3) * ldc + 2 * i + m % 3;
            zx[m] = __ldcg(uc + k);
            zy[m] = __ldcg(uc + n2c + k);
        }
        const int o = orient(i, j, nc);
#pragma unroll
        for (int fb = 0; fb < 4; ++fb)
#pragma unroll
            for (int fa = 0; fa < 4; ++fa) {
                const int X = 4 * i + fa, Y = 4 * j + fb;
                if (!interior2(X, Y, nf)) continue;
                float sx = 0.f, sy = 0.f;
#pragma unroll
                for (int L = 0; L < 9; ++L) {
                    const float w = wt.w[o][L][fb][fa];
                    sx = fmaf(w, zx[L], sx);
                    sy = fmaf(w, zy[L], sy);
                }
                const int k = Y * ldf + X;
                u[k] = __ldcg(u + k) + sx;
                u[n2f + k] = __ldcg(u + n2f + k) + sy;
            }
    }
    auto P = [&](int a, int b) { return __ldcg(pc + b * (nc + 1) + a); };
    auto add = [&](int x, int y, float v) { p[y * (nf + 1) + x] = __ldcg(p + y * (nf + 1) + x) + v; };
    const float p00 = P(i, j);
    add(2 * i, 2 * j, p00);
    if (i < nc) add(2 * i + 1, 2 * j, 0.5f * (p00 + P(i + 1, j)));
    if (j < nc) add(2 * i, 2 * j + 1, 0.5f * (p00 + P(i, j + 1)));
    if (i < nc && j < nc) add(2 * i + 1, 2 * j + 1, 0.5f * (orient(i, j, nc) == 0 ? p00 + P(i + 1, j + 1) : P(i + 1, j) + P(i, j + 1)));
}

// The exact solve on the coarsest level c of the iteration into its (u, p): c = 0 with the 27 x 27
// bordered inverse, c > 0 with the dense bordered inverse (rows over every warp of the grid, the
// right-hand side gathered into each CTA's shared memory F).
__device__ void small_coarse_solve(const SmallCycleArgs& A, double* F) {
    const SmallLevelArgs& Z = A.L[A.clev];
    const int n = 2 << A.clev, ld = 2 * n + 1, n2 = ld * ld, nm = 2 * n - 1, nv = nm * nm;
    const int nunk = A.clev == 0 ? 27 : A.cnb - 1;
    const double* inv = A.clev == 0 ? A.inv0 : A.cinv;
    const int stride = A.clev == 0 ? 27 : A.cnb;
    for (int t = threadIdx.x; t < nunk; t += blockDim.x) {
        double v;
        if (t < 2 * nv) {
            const int c = t / nv, r = t - c * nv;
            v = (double)__ldcg(Z.f + c * n2 + (r / nm + 1) * ld + r % nm + 1);
        } else {
            v = (double)__ldcg(Z.g + (t - 2 * nv));
        }
        F[t] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < nunk; row += nwarps) {
        const double* r = inv + (size_t)row * stride;
        double acc = 0.0;
#pragma unroll 8
        for (int j = lane; j < nunk; j += 32) acc = fma(__ldg(r + j), F[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            if (row < 2 * nv) {
                const int c = row / nv, q = row - c * nv;
                Z.u[c * n2 + (q / nm + 1) * ld + q % nm + 1] = (float)acc;
            } else {
                Z.p[row - 2 * nv] = (float)acc;
            }
        }
    }
}

__global__ void __launch_bounds__(32 * kSmallNW, 1) k_small_cycle(const __grid_constant__ SmallCycleArgs A) {
    using G = TmaTile;
    constexpr int TY = kSmallTY;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float2* sU = reinterpret_cast<float2*>(base + 128);
    float2* sF = reinterpret_cast<float2*>(base + G::off_f(TY));
    float* sP = reinterpret_cast<float*>(base + G::off_p(TY));
    float* sG = reinterpret_cast<float*>(base + G::off_g(TY));
    float* sS = reinterpret_cast<float*>(base + G::off_s(TY));
    double* sRhs = reinterpret_cast<double*>(base + G::bytes(TY));            // coarsest right-hand side
    OpCoef<float>* sc = reinterpret_cast<OpCoef<float>*>(sRhs + kSmallMaxNb);  // levels clev + 1 .. top
    const int nlev = A.top - A.clev;
    {
        const float* src = reinterpret_cast<const float*>(A.coef + A.clev + 1);
        float* dst = reinterpret_cast<float*>(sc);
        const int words = nlev * (int)(sizeof(OpCoef<float>) / sizeof(float));
        for (int t = threadIdx.x; t < words; t += blockDim.x) dst[t] = __ldg(src + t);
    }
    __syncthreads();
    unsigned k = 0;                // grid barriers passed
    bool sw[kSmallTop + 1] = {};   // level state in (tu, tp) instead of (u, p)
    int cnt[kSmallTop + 1] = {};   // coarse corrections still to do at a level
    int l = A.top;
    bool enter = true;
    auto tiles = [&](int n, int& cols) {
        cols = (n + 1 + G::TX - 1) / G::TX;
        return cols * ((n + 1 + TY - 1) / TY);
    };
    auto smooth = [&](int lv) {   // one Uzawa step on level lv, ping-pong
        const SmallLevelArgs& L = A.L[lv];
        const int n = 2 << lv;
        const float* xu = sw[lv] ? L.tu : L.u;
        const float* xp = sw[lv] ? L.tp : L.p;
        float* ou = sw[lv] ? L.u : L.tu;
        float* op = sw[lv] ? L.p : L.tp;
        int cols;
        const int nt = tiles(n, cols);
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const int i0 = (t % cols) * G::TX, j0 = (t / cols) * TY;
            stage_compact(n, TY, i0, j0, j0 - 1, xu, xp, L.f, L.g, L.sinv, sU, sF, sP, sG, sS);
            __syncthreads();
            reg_phases<G, false, kSmallNW>(n, TY, i0, j0, sc[lv - A.clev - 1], A.q[lv], A.tau, A.sigma, sU, sF, sP, sG,
                                           sS, ou, op);
            __syncthreads();
        }
        sw[lv] = !sw[lv];
        return grid_barrier(A.bar, ++k);
    };
    while (true) {
        if (enter) {
            if (l == A.clev) {
                small_coarse_solve(A, sRhs);
                sw[l] = false;
                if (!grid_barrier(A.bar, ++k)) return;
                enter = false;
                continue;
            }
            for (int m = 0; m < A.nu_pre; ++m)
                if (!smooth(l)) return;
            {   // defect and restriction into level l - 1, whose iterate starts from zero
                const SmallLevelArgs& L = A.L[l];
                const SmallLevelArgs& C = A.L[l - 1];
                const int n = 2 << l;
                int cols;
                const int nt = tiles(n, cols);
                for (int t = blockIdx.x; t < nt; t += gridDim.x) {
                    const int i0 = (t % cols) * G::TX, j0 = (t / cols) * TY;
                    stage_compact(n, TY, i0, j0, j0 - 2, sw[l] ? L.tu : L.u, sw[l] ? L.tp : L.p, L.f, L.g, nullptr, sU,
                                  sF, sP, sG, sS);
                    __syncthreads();
                    defect_restrict<G, kSmallNW, false>(n, TY, i0, j0, sc[l - A.clev - 1], A.q[l], A.wt, sU, sF, sP, sG,
                                                        C.f, C.g, C.u, C.p);
                    __syncthreads();
                }
                sw[l - 1] = false;
                if (!grid_barrier(A.bar, ++k)) return;
            }
            cnt[l] = A.gamma;
            --l;
        } else {
            if (l == A.top) break;
            const int pl = l + 1;
            if (--cnt[pl] > 0) {   // the W-cycle's next coarse correction, from the current coarse iterate
                l = pl - 1;
                enter = true;
                continue;
            }
            {   // prolongation and correction
                const SmallLevelArgs& C = A.L[l];
                const SmallLevelArgs& L = A.L[pl];
                const int nc = 2 << l, cells = (nc + 1) * (nc + 1);
                const float* uc = sw[l] ? C.tu : C.u;
                const float* pc = sw[l] ? C.tp : C.p;
                float* uf = sw[pl] ? L.tu : L.u;
                float* pf = sw[pl] ? L.tp : L.p;
                for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cells; q += gridDim.x * blockDim.x)
                    small_prolong_cell(q % (nc + 1), q / (nc + 1), nc, A.wt, uc, pc, uf, pf);
                if (!grid_barrier(A.bar, ++k)) return;
            }
            for (int m = 0; m < A.nu_post; ++m)
                if (!smooth(pl)) return;
            l = pl;
        }
    }
    if (sw[A.top]) {   // odd number of steps on the top level: its state back to (u, p)
        const SmallLevelArgs& L = A.L[A.top];
        const int n = 2 << A.top, nu = 2 * (2 * n + 1) * (2 * n + 1), np = (n + 1) * (n + 1);
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nu; q += gridDim.x * blockDim.x) L.u[q] = __ldcg(L.tu + q);
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) L.p[q] = __ldcg(L.tp + q);
    }
}

// dynamic shared memory: the tiles, the coarsest right-hand side, nlev levels' operators, and the
// slack that aligns the base to 128 bytes
size_t small_cycle_smem(int nlev) {
    return TmaTile::bytes(kSmallTY) + sizeof(double) * kSmallMaxNb + sizeof(OpCoef<float>) * (size_t)nlev + 128;
}

template <int NW, int MINB>
cudaError_t reg_smem_attr() {
    return cudaFuncSetAttribute(k_uzawa_reg<NW, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RegTile::bytes(kRegMaxRows));
}
template <int NW, int MINB, bool PAIR = false>
cudaError_t tma_smem_attr() {
    return cudaFuncSetAttribute(k_uzawa_tma<NW, MINB, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TmaTile::bytes(kRegMaxRows));
}

// Rows per tile for level size n: the least work on the busiest SM, (tiles per SM, rounded up) x
// (work of one tile, about ty + 4 rows of the u^{m-1/2} region), among the tile heights that keep
// at least MINB CTAs of kernel k (dynamic shared memory G::bytes(ty)) resident per SM.
template <class G, class K>
int tile_rows(int n, K k, int nthreads, int minb, int* cache, bool even = false) {
    const int lv = 31 - __builtin_clz((unsigned)n);
    int& r = cache[lv & 31];
    if (r) return r;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::max(sms, 1);
    const int cols = (n + 1 + G::TX - 1) / G::TX;
    double best = 1e300;
    int best_ty = 12;
    for (int ty = 4; ty <= kRegMaxRows; ty += even ? 2 : 1) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nthreads, G::bytes(ty)) != cudaSuccess ||
            per_sm < minb)
            continue;
        const long tiles = (long)cols * ((n + 1 + ty - 1) / ty);
        const double cost = (double)((tiles + sms - 1) / sms) * (ty + 4);
        if (cost < best) {
            best = cost;
            best_ty = ty;
        }
    }
    cudaGetLastError();
    r = best_ty;
    return r;
}

template <bool PC>
cudaError_t rt_smem_attr() {
    return cudaFuncSetAttribute(k_restrict_tma<8, 3, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TmaTile::bytes(kRegMaxRows));
}

template <int NW, int MINB>
int reg_rows(int n) {
    static int cache[32] = {};
    return tile_rows<RegTile>(n, k_uzawa_reg<NW, MINB>, 32 * NW, MINB, cache);
}
template <int NW, int MINB, bool PAIR = false>
int tma_rows(int n) {
    static int cache[32] = {};
    return tile_rows<TmaTile>(n, k_uzawa_tma<NW, MINB, PAIR>, 32 * NW, MINB, cache, PAIR);
}
template <class G>
TileOrder tile_order(int n, int ty) {
    TileOrder ord;
    ord.cols = (n + 1 + G::TX - 1) / G::TX;
    ord.rows = (n + 1 + ty - 1) / ty;
    mid_band(n / 2, G::TX, ord.cols, ord.c0, ord.nc);
    mid_band(n / 2, ty, ord.rows, ord.r0, ord.nr);
    return ord;
}

template <int NW, int MINB>
bool launch_reg_v(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, const float* u, const float* p,
                  const float* f, const float* g, const float* sinv, float* u_out, float* p_out) {
    RegCoef q;
    if (!make_reg_coef(c, tau, q)) return false;
    const int ty = reg_rows<NW, MINB>(n);
    const TileOrder ord = tile_order<RegTile>(n, ty);
    launch_pdl(k_uzawa_reg<NW, MINB>, dim3(ord.cols * ord.rows), dim3(32 * NW), RegTile::bytes(ty), s, n, ty, ord, c, q, tau,
               sigma, u, p, f, g, sinv, u_out, p_out);
    return true;
}

// cuTensorMapEncodeTiled, from the driver through the runtime's entry-point query (no link to the
// driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
            qr != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// float32 box map over `rank` dimensions (strides in bytes for dimensions 1..rank-1), zero fill
bool encode_box(CUtensorMap& m, const float* base, cuuint32_t rank, const cuuint64_t* dims, const cuuint64_t* strides,
                const cuuint32_t* box) {
    const cuuint32_t es[3] = {1, 1, 1};
    return encode_tiled()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tile maps of a planar level with N = n, tile height ty
bool make_tma_maps(int n, int ty, const float* u, const float* p, const float* f, const float* g, const float* sinv,
                   TmaMaps& m) {
    if (!encode_tiled()) return false;
    const cuuint64_t P = (cuuint64_t)pl_pitch(n), RP = (cuuint64_t)pl_rows(n), VP = (cuuint64_t)pl_vpitch(n);
    const cuuint64_t rows = (cuuint64_t)n + 1;
    const cuuint64_t ud[3] = {2 * P, RP, 2}, us[2] = {8 * P, 8 * P * RP};
    const cuuint32_t ub[3] = {2 * TmaTile::UWH, (cuuint32_t)(2 * (ty + 6)), 2};
    const cuuint64_t fd[3] = {2 * P, rows, 2}, fs[2] = {16 * P, 8 * P * RP};
    const cuuint32_t fb[3] = {2 * TmaTile::FW, (cuuint32_t)(ty + 4), 2};
    const cuuint64_t vd[2] = {VP, rows}, vs[1] = {4 * VP};
    const cuuint32_t pb[2] = {TmaTile::PW, (cuuint32_t)(ty + 6)}, gb[2] = {TmaTile::DW, (cuuint32_t)(ty + 2)};
    return encode_box(m.u, u, 3, ud, us, ub) && encode_box(m.f0, f, 3, fd, fs, fb) &&
           encode_box(m.f1, f + 2 * P, 3, fd, fs, fb) && encode_box(m.p, p, 2, vd, vs, pb) &&
           encode_box(m.g, g, 2, vd, vs, gb) && encode_box(m.s, sinv, 2, vd, vs, gb);
}

template <int NW, int MINB, bool PAIR = false>
bool launch_tma_v(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, const float* u, const float* p,
                  const float* f, const float* g, const float* sinv, float* u_out, float* p_out, bool prefetch,
                  const CoarseCorrection& cc) {
    RegCoef q;
    if (!make_reg_coef(c, tau, q)) return false;
    int ty = tma_rows<NW, MINB, PAIR>(n);
    if (cc.u) ty = std::min(ty, kEmbedMaxRows);
    TmaMaps m;
    if (!make_tma_maps(n, ty, u, p, f, g, sinv, m)) return false;
    const TileOrder ord = tile_order<TmaTile>(n, ty);
    int pf = 0;
    if (prefetch) {   // one wave of resident CTAs ahead
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_uzawa_tma<NW, MINB, PAIR>, 32 * NW,
                                                          TmaTile::bytes(ty)) != cudaSuccess)
            per_sm = MINB;
        cudaGetLastError();
        pf = std::max(1, sms) * std::max(1, per_sm);
    }
    launch_pdl(k_uzawa_tma<NW, MINB, PAIR>, dim3(ord.cols * ord.rows), dim3(32 * NW), TmaTile::bytes(ty), s, n, ty, ord, c,
               q, tau, sigma, m, u_out, p_out, pf, cc.u, cc.p, cc.planar ? 1 : 0);
    return true;
}

// the compile-time embedding table equals the host element code's transfer weights
bool embed_table_matches() {
    static const bool ok = [] {
        const TransferWeights t = transfer_weights();
        for (int o = 0; o < 2; ++o)
            for (int L = 0; L < 9; ++L)
                for (int fb = 0; fb < 4; ++fb)
                    for (int fa = 0; fa < 4; ++fa)
                        if (std::fabs(t.P2[o][L][fb][fa] - embed_weight(o, L, fa, fb)) > 1e-14) return false;
        return true;
    }();
    return ok;
}

const RestrictWeights& restrict_weights() {
    static const RestrictWeights w = [] {
        RestrictWeights r{};
        const TransferWeights t = transfer_weights();
        for (int o = 0; o < 2; ++o)
            for (int L = 0; L < 9; ++L)
                for (int fb = 0; fb < 4; ++fb)
                    for (int fa = 0; fa < 4; ++fa) r.w[o][L][fb][fa] = (float)t.P2[o][L][fb][fa];
        return r;
    }();
    return w;
}

template <bool PC>
bool launch_rt(cudaStream_t s, int n, const OpCoef<float>& c, const float* u, const float* p, const float* f,
               const float* g, float* fc, float* gc, float* uc, float* pc) {
    RegCoef q;
    if (!make_reg_coef(c, 1.0f, q)) return false;
    const int ty = std::max(4, tma_rows<8, 3>(n) & ~1);   // even: whole coarse cells per tile
    TmaMaps m;
    if (!make_tma_maps(n, ty, u, p, f, g, g, m)) return false;   // no Shat^{-1} tile (its map is unused)
    const TileOrder ord = tile_order<TmaTile>(n, ty);
    launch_pdl(k_restrict_tma<8, 3, PC>, dim3(ord.cols * ord.rows), dim3(256), TmaTile::bytes(ty), s, n, ty, ord, c, q,
               restrict_weights(), m, fc, gc, uc, pc);
    return true;
}

cudaError_t small_smem_attr() {
    return cudaFuncSetAttribute(k_small_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)small_cycle_smem(kSmallTop));
}

}  // namespace

cudaError_t launch_small_cycle(cudaStream_t s, const SmallCycleHost& h) {
    if (h.top < 1 || h.top > kSmallTop || h.clev < 0 || h.clev >= h.top || h.cnb > kSmallMaxNb) return cudaErrorInvalidValue;
    SmallCycleArgs A{};
    for (int l = h.clev; l <= h.top; ++l) {
        A.L[l] = SmallLevelArgs{h.u[l], h.p[l], h.f[l], h.g[l], h.tu[l], h.tp[l], h.sinv[l]};
        if (l > h.clev && !make_reg_coef(*h.coef_host[l], h.tau, A.q[l])) return cudaErrorInvalidValue;
    }
    A.coef = h.coef_dev;
    A.wt = restrict_weights();
    A.inv0 = h.inv0;
    A.cinv = h.cinv;
    A.cnb = h.cnb;
    A.bar = h.bar;
    A.tau = h.tau;
    A.sigma = h.sigma;
    A.nu_pre = h.nu_pre;
    A.nu_post = h.nu_post;
    A.gamma = h.gamma;
    A.top = h.top;
    A.clev = h.clev;
    const size_t smem = small_cycle_smem(h.top - h.clev);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_cycle, 32 * kSmallNW, smem);
    if (e != cudaSuccess) return e;
    // every SM: the tile phases use at most `tiles` CTAs, the coarsest solve's rows all of them
    const int grid = std::max(1, sms * per_sm);
    if ((e = cudaMemsetAsync(h.bar, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * kSmallNW);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: the grid barriers complete
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_small_cycle, A);
}

bool launch_restrict_tma(cudaStream_t s, int n, bool pc_planar, const OpCoef<float>& c, const float* u, const float* p,
                         const float* f, const float* g, float* fc, float* gc, float* uc, float* pc) {
    return pc_planar ? launch_rt<true>(s, n, c, u, p, f, g, fc, gc, uc, pc)
                     : launch_rt<false>(s, n, c, u, p, f, g, fc, gc, uc, pc);
}

cudaError_t prepare_uzawa_reg() {
    cudaError_t e = reg_smem_attr<8, 2>();
    if (e == cudaSuccess) e = reg_smem_attr<8, 4>();
    if (e == cudaSuccess) e = tma_smem_attr<8, 3>();
    if (e == cudaSuccess) e = tma_smem_attr<8, 4>();
    if (e == cudaSuccess) e = tma_smem_attr<8, 2, true>();
    if (e == cudaSuccess) e = tma_smem_attr<8, 3, true>();
    if (e == cudaSuccess) e = rt_smem_attr<true>();
    if (e == cudaSuccess) e = rt_smem_attr<false>();
    if (e == cudaSuccess) e = small_smem_attr();
    return e;
}

bool launch_uzawa_reg(int variant, cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma,
                      const float* u, const float* p, const float* f, const float* g, const float* sinv,
                      float* u_out, float* p_out) {
    if (variant == 0) return launch_reg_v<8, 2>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
    return launch_reg_v<8, 4>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
}

namespace {
int g_tma_choice[32] = {};     // planar step variant per level size (log2 N)
bool g_tma_tuned[32] = {};
int lvl(int n) { return (31 - __builtin_clz((unsigned)n)) & 31; }
}  // namespace

bool launch_uzawa_tma_variant(int variant, cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma,
                              const float* u, const float* p, const float* f, const float* g, const float* sinv,
                              float* u_out, float* p_out, const CoarseCorrection& cc) {
    if (cc.u && (!cc.p || !embed_table_matches())) return false;
    switch (variant) {
        case 1: return launch_tma_v<8, 3>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, true, cc);
        case 2: return launch_tma_v<8, 4>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, false, cc);
        case 3: return launch_tma_v<8, 4>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, true, cc);
        case 4: return launch_tma_v<8, 2, true>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, true, cc);
        case 5: return launch_tma_v<8, 3, true>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, true, cc);
        default: return launch_tma_v<8, 3>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, false, cc);
    }
}

bool launch_uzawa_tma(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, const float* u,
                      const float* p, const float* f, const float* g, const float* sinv, float* u_out, float* p_out,
                      const CoarseCorrection& cc) {
    return launch_uzawa_tma_variant(g_tma_choice[lvl(n)], s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, cc);
}

bool uzawa_tma_embed_available() { return uzawa_tma_available() && embed_table_matches(); }

void embed_weights_table(double* w) {
    for (int o = 0; o < 2; ++o)
        for (int L = 0; L < 9; ++L)
            for (int fb = 0; fb < 4; ++fb)
                for (int fa = 0; fa < 4; ++fa) w[((o * 9 + L) * 4 + fb) * 4 + fa] = embed_weight(o, L, fa, fb);
}

int tma_choice(int n) { return g_tma_choice[lvl(n)]; }
bool tma_tuned(int n) { return g_tma_tuned[lvl(n)]; }
bool set_tma_choice(int n, int v) {
    if (v < 0 || v >= kTmaVariants) return false;
    g_tma_choice[lvl(n)] = v;
    g_tma_tuned[lvl(n)] = true;
    return true;
}

cudaError_t autotune_uzawa_tma(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, float* u,
                               float* p, const float* f, const float* g, const float* sinv, float* u_out, float* p_out) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cudaErrorUnknown;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cudaErrorUnknown;
    }
    const int reps = n >= 512 ? 5 : 20;
    int best = 0;
    float bms = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int v = 0; v < kTmaVariants && err == cudaSuccess; ++v) {
        if (!launch_uzawa_tma_variant(v, s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out)) continue;   // warm-up
        bool sw = true;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r) {
            launch_uzawa_tma_variant(v, s, n, c, tau, sigma, sw ? u_out : u, sw ? p_out : p, f, g, sinv, sw ? u : u_out,
                                     sw ? p : p_out);
            sw = !sw;
        }
        cudaEventRecord(e1, s);
        if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < bms) {
            bms = ms / reps;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    g_tma_choice[lvl(n)] = best;
    g_tma_tuned[lvl(n)] = true;
    return cudaGetLastError();
}

bool uzawa_tma_available() { return encode_tiled() != nullptr; }

unsigned uzawa_tma_timeouts() {
    unsigned v = 0;
    const unsigned zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_tma_timeout, sizeof v) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_tma_timeout, &zero, sizeof zero);
    return v;
}

}  // namespace smg
