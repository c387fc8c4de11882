// uzawa_pair.cu -- the float32 Uzawa step (Sec. 4) in one kernel, with the two velocity
// components of every lattice point side by side in shared memory and packed FP32x2 arithmetic.
//
//   u^{m-1/2} = u^{m-1} + tau Ahat^{-1} (f - A u^{m-1} - B^T p^{m-1})
//   dp        = sigma Shat^{-1} (B u^{m-1/2} - g),      p^{m} = p^{m-1} + dp
//   u^{m}     = u^{m-1/2} - tau Ahat^{-1} B^T dp
//
// The velocity block of the operator acts on both components with the same coefficients, and B,
// B^T pair an x and a y coefficient with one value, so with (u_x, u_y) stored as one float2 a row
// term is one 64-bit shared load and one packed fused multiply-add (FFMA2) for both components.
//
// A CTA owns a 28 x ty tile of cells; its NW warps stage u and p with a three-cell halo, compute
// u^{m-1/2} on the tile plus two cells (32 cells per row: one row per warp pass), dp on the tile
// plus one vertex, and the new (u, p) on the tile.  Tiles away from the two mid-lines (all but a
// few) take a path with every structural test decided at compile time for the tile's one stencil
// class (at the boundary the zero-filled halo stands for the Dirichlet values, and only unknowns
// are written); the tiles at the mid-lines run the general merged-stencil rows of cellops.cuh, cell
// by cell, on the same shared tiles.
#include <algorithm>

#include "cellops.cuh"
#include "kernels.cuh"
#include "tiles.cuh"

namespace smg {

// merged-stencil coefficients of the two orientation classes as component pairs
struct PairCoef {
    float2 MA[2][4][25];   // (a, a): row coefficient of node s applied to (u_x, u_y)
    float2 MBT[2][4][9];   // (B^T_x, B^T_y) of node s applied to (p, p)
    float2 MB[2][25];      // (B_x, B_y) applied to (u_x, u_y); the row value is the sum of both
    float TI[2][4];        // tau / diag A of node s
};

static PairCoef make_pair_coef(const OpCoef<float>& c, float tau) {
    PairCoef q{};
    for (int k = 0; k < 2; ++k) {
        for (int s = 0; s < 4; ++s) {
            for (int w = 0; w < 25; ++w) q.MA[k][s][w] = make_float2(c.MA[k][s][w], c.MA[k][s][w]);
            for (int v = 0; v < 9; ++v) q.MBT[k][s][v] = make_float2(c.MBTx[k][s][v], c.MBTy[k][s][v]);
            q.TI[k][s] = tau * c.MIdg[k][s];
        }
        for (int w = 0; w < 25; ++w) q.MB[k][w] = make_float2(c.MBx[k][w], c.MBy[k][w]);
    }
    return q;
}

// Tile geometry for TX = 28 columns of cells and a run-time number of rows ty (chosen per level
// so that the tiles fill whole waves of resident CTAs, see pair_rows).
struct PairTile {
    static constexpr int TX = 28;
    static_assert(TX + 4 == 32, "one warp covers a row of the u^{m-1/2} region");
    // u: cells [i0-3, i0+TX+3) x [j0-3, j0+ty+3); lattice columns split by parity into two planes
    static constexpr int UWH = TX + 6;   // float2 per plane row
    // u^{m-1/2}: cells [i0-2, i0+TX+2) x [j0-2, j0+ty+2)
    static constexpr int HWH = TX + 4;
    static constexpr int PW = TX + 6;    // p: vertices [i0-3, i0+TX+3)
    static constexpr int DW = TX + 2;    // dp: vertices [i0-1, i0+TX+1)
    __host__ __device__ static constexpr int upl(int ty) { return UWH * 2 * (ty + 6); }
    __host__ __device__ static constexpr int hpl(int ty) { return HWH * 2 * (ty + 4); }
    __host__ __device__ static constexpr size_t bytes(int ty) {
        return 8 * (size_t)(2 * upl(ty) + 2 * hpl(ty)) + 4 * (size_t)(PW * (ty + 6) + DW * (ty + 2));
    }
};
constexpr int kPairMaxRows = 20;

// One component of a float2 lattice tile (general path; same addressing as SLat).  The component
// is a member so that both views share one type; it is a constant wherever a view is built.
template <int WH>
struct PairLat {
    static constexpr bool zero_filled = true;
    const float2* p;
    int pl;        // float2 per parity plane
    int xh0, y0;   // tile origin: X0 = 2 xh0, Y0 = y0
    bool ycomp;
    __device__ __forceinline__ float at(int si, int sj, int a, int b) const {
        const float2 e = p[(a & 1) * pl + (2 * sj + b - y0) * WH + (si - xh0) + (a >> 1)];
        return ycomp ? e.y : e.x;
    }
    __device__ __forceinline__ float operator()(int X, int Y) const {
        const int dx = X - 2 * xh0;
        const float2 e = p[(dx & 1) * pl + (Y - y0) * WH + (dx >> 1)];
        return ycomp ? e.y : e.x;
    }
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// ---- fast path (class C, every node an unknown, every window inside the tile)
// window point W (5 x 5 around the cell's vertex) of a float2 lattice tile; `b` addresses the cell
// t0 / t1: the cell's position in the even / odd parity plane
template <int WH, int W>
__device__ __forceinline__ float2 win2(const float2* t0, const float2* t1) {
    constexpr int dx = W % 5 - 2, dy = W / 5 - 2;
    return ((dx & 1) ? t1 : t0)[dy * WH + (dx >> 1)];
}

template <int C, int S, int W>
__device__ __forceinline__ void ma_pair(const PairCoef& q, float2 w, float2 (&au)[4]) {
    if constexpr (nz_MA(C, S, W)) au[S] = __ffma2_rn(q.MA[C][S][W], w, au[S]);
}
template <int C, int WH, int W>
__device__ __forceinline__ void phase1_w(const PairCoef& q, const float2* t0, const float2* t1, float2 (&au)[4],
                                         float2 (&ctr)[4]) {
    if constexpr (need_win(C, true, false, W)) {
        const float2 w = win2<WH, W>(t0, t1);
        ma_pair<C, 0, W>(q, w, au);
        ma_pair<C, 1, W>(q, w, au);
        ma_pair<C, 2, W>(q, w, au);
        ma_pair<C, 3, W>(q, w, au);
        // the owned nodes V, H, E, C sit at window points 12, 13, 17, 18
        if constexpr (W == 12) ctr[0] = w;
        if constexpr (W == 13) ctr[1] = w;
        if constexpr (W == 17) ctr[2] = w;
        if constexpr (W == 18) ctr[3] = w;
    }
}
template <int C, int S, int V>
__device__ __forceinline__ void mbt_pair(const PairCoef& q, float2 pv, float2 (&bt)[4]) {
    if constexpr (nz_MBT(C, S, V)) bt[S] = __ffma2_rn(q.MBT[C][S][V], pv, bt[S]);
}
template <int C, int PW, int V>
__device__ __forceinline__ void bt_v(const PairCoef& q, const float* sp, int b, float2 (&bt)[4]) {
    if constexpr (need_vwin(C, V)) {
        const float v = sp[b + (V / 3 - 1) * PW + V % 3 - 1];
        const float2 pv = f2(v, v);
        mbt_pair<C, 0, V>(q, pv, bt);
        mbt_pair<C, 1, V>(q, pv, bt);
        mbt_pair<C, 2, V>(q, pv, bt);
        mbt_pair<C, 3, V>(q, pv, bt);
    }
}
template <int C, int PW, int... V>
__device__ __forceinline__ void bt_rows(const PairCoef& q, const float* sp, int b, float2 (&bt)[4],
                                        std::integer_sequence<int, V...>) {
    (bt_v<C, PW, V>(q, sp, b, bt), ...);
}
template <int C, int WH, int... W>
__device__ __forceinline__ void a_rows(const PairCoef& q, const float2* t0, const float2* t1, float2 (&au)[4],
                                       float2 (&ctr)[4], std::integer_sequence<int, W...>) {
    (phase1_w<C, WH, W>(q, t0, t1, au, ctr), ...);
}
template <int C, int WH, int W>
__device__ __forceinline__ void b_w(const PairCoef& q, const float2* t0, const float2* t1, float2& acc) {
    if constexpr (nz_MB(C, W)) acc = __ffma2_rn(q.MB[C][W], win2<WH, W>(t0, t1), acc);
}
template <int C, int WH, int... W>
__device__ __forceinline__ float b_row(const PairCoef& q, const float2* t0, const float2* t1,
                                       std::integer_sequence<int, W...>) {
    float2 acc = f2(0.f, 0.f);
    (b_w<C, WH, W>(q, t0, t1, acc), ...);
    return acc.x + acc.y;
}

template <int NW>
__global__ void __launch_bounds__(32 * NW, (NW > 8 ? 2 : NW > 4 ? 3 : 6))
    k_uzawa_pair(int n, int TY, TileOrder ord, const __grid_constant__ OpCoef<float> c, const __grid_constant__ PairCoef q, float tau,
                 float sigma, const float* __restrict__ u, const float* __restrict__ p, const float* __restrict__ f,
                 const float* __restrict__ g, const float* __restrict__ sinv, float* __restrict__ u_out,
                 float* __restrict__ p_out) {
    pdl_wait();
    using G = PairTile;
    constexpr int TX = G::TX;
    const int UPL = G::upl(TY), HPL = G::hpl(TY);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sU = reinterpret_cast<float2*>(smem_raw);
    float2* sH = sU + 2 * UPL;
    float* sP = reinterpret_cast<float*>(sH + 2 * HPL);
    float* sD = sP + G::PW * (TY + 6);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int tc, tr;
    ord.tile(blockIdx.x, tc, tr);
    const int i0 = tc * TX, j0 = tr * TY;
    const int ld = 2 * n + 1, n2 = ld * ld, h = n >> 1;
    // fast: the u^{m-1/2} region is off the mid-lines, so every cell of the tile has the stencil
    // class of its quadrant; inner: besides, the staged region lies strictly inside the domain, so
    // nothing needs a range test or a Dirichlet mask
    const bool fast = (h < i0 - 2 || h >= i0 + TX + 2) && (h < j0 - 2 || h >= j0 + TY + 2);
    const bool inner = fast && i0 >= 4 && j0 >= 4 && i0 + TX + 3 <= n && j0 + TY + 3 <= n;
    const int cls = orient(i0, j0, n);

    // ---- stage u as (u_x, u_y) pairs and p; zero outside the domain and on its boundary
    // A lane stages lattice columns x = lane + 32 t of every row it takes: the parity plane
    // (lane & 1) and the plane column (lane >> 1) + 16 t are fixed per lane, so a row costs one
    // address computation and the loads and stores use constant offsets from it.
    const int X0 = 2 * (i0 - 3), Y0 = 2 * (j0 - 3);
    static_assert(2 * G::UWH == 68 && G::PW == 34, "staging loops below assume 68 lattice columns, 34 vertices");
    {
        float2* srow = sU + (lane & 1) * UPL + (lane >> 1);
        for (int y = warp; y < 2 * (TY + 6); y += NW) {
            const int Y = Y0 + y;
            const int k = Y * ld + X0 + lane;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (t == 2 && lane >= 4) break;
                float2 v = f2(0.f, 0.f);
                if (inner || interior2(X0 + lane + 32 * t, Y, n)) v = f2(__ldg(u + k + 32 * t), __ldg(u + n2 + k + 32 * t));
                srow[y * G::UWH + 16 * t] = v;
            }
        }
    }
    for (int y = warp; y < TY + 6; y += NW) {
        const int J = j0 - 3 + y;
        const int k = J * (n + 1) + i0 - 3 + lane;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (t == 1 && lane >= 2) break;
            const int I = i0 - 3 + lane + 32 * t;
            sP[y * G::PW + lane + 32 * t] =
                (inner || (I >= 0 && J >= 0 && I <= n && J <= n)) ? __ldg(p + k + 32 * t) : 0.f;
        }
    }
    __syncthreads();

    using UL = PairLat<G::UWH>;
    using HL = PairLat<G::HWH>;

    // ---- u^{m-1/2} on cells (i0 - 2 + lane, j0 - 2 + r)
    for (int r = warp; r < TY + 4; r += NW) {
        const int ci = i0 - 2 + lane, cj = j0 - 2 + r;
        float2 hv[4];
        if (fast) {
            float2 au[4], bt[4], ctr[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) au[s] = bt[s] = ctr[s] = f2(0.f, 0.f);
            const float2* t0 = sU + 2 * (r + 1) * G::UWH + lane + 1;
            const float2* t1 = t0 + UPL;
            const int bp = (r + 1) * G::PW + lane + 1;
            if (cls == 0) {
                a_rows<0, G::UWH>(q, t0, t1, au, ctr, std::make_integer_sequence<int, 25>{});
                bt_rows<0, G::PW>(q, sP, bp, bt, std::make_integer_sequence<int, 9>{});
            } else {
                a_rows<1, G::UWH>(q, t0, t1, au, ctr, std::make_integer_sequence<int, 25>{});
                bt_rows<1, G::PW>(q, sP, bp, bt, std::make_integer_sequence<int, 9>{});
            }
            // on a tile at the boundary the rows are the same (the staged zeros stand for the
            // Dirichlet values and for everything outside); only unknowns keep their value
            const bool ci_in = ci > 0 && ci < n, cj_in = cj > 0 && cj < n;
            const bool ci_h = ci >= 0 && ci < n, cj_h = cj >= 0 && cj < n;
            const bool unk[4] = {inner || (ci_in && cj_in), inner || (ci_h && cj_in), inner || (ci_in && cj_h),
                                 inner || (ci_h && cj_h)};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                hv[s] = f2(0.f, 0.f);
                if (unk[s]) {
                    const int k = (2 * cj + (s >> 1)) * ld + 2 * ci + (s & 1);
                    const float2 fs = f2(__ldg(f + k), __ldg(f + n2 + k));
                    const float ti = q.TI[cls][s];
                    hv[s] = __ffma2_rn(f2(ti, ti), f2(fs.x - au[s].x - bt[s].x, fs.y - au[s].y - bt[s].y), ctr[s]);
                }
            }
        } else {
#pragma unroll
            for (int s = 0; s < 4; ++s) hv[s] = f2(0.f, 0.f);
            if (ci >= 0 && cj >= 0 && ci <= n && cj <= n) {
                const UL vux{sU, UPL, i0 - 3, Y0, false};
                const UL vuy{sU, UPL, i0 - 3, Y0, true};
                const SVert<float, G::PW> vp{sP, i0 - 3, j0 - 3};
                Acc<float> a;
                cell_apply_auto<true, true, false, true, false>(ci, cj, n, c, vux, vuy, vp, a);
                const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    if (!slot_unknown(cn, s)) continue;
                    const int k = (2 * cj + (s >> 1)) * ld + 2 * ci + (s & 1);
                    const float w = tau * a.idg[s];
                    hv[s] = f2(vux.at(ci, cj, s & 1, s >> 1) + w * (__ldg(f + k) - a.au[0][s] - a.bt[0][s]),
                               vuy.at(ci, cj, s & 1, s >> 1) + w * (__ldg(f + n2 + k) - a.au[1][s] - a.bt[1][s]));
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) sH[(s & 1) * HPL + (2 * r + (s >> 1)) * G::HWH + lane] = hv[s];
    }
    __syncthreads();

    // ---- dp on vertices (i0 - 1 + lane, j0 - 1 + r), lane < TX + 2
    for (int r = warp; r < TY + 2; r += NW) {
        if (lane >= TX + 2) break;
        const int vi = i0 - 1 + lane, vj = j0 - 1 + r;
        float d = 0.f;
        if (fast && (inner || (vi >= 0 && vj >= 0 && vi <= n && vj <= n))) {
            const float2* t0 = sH + 2 * (r + 1) * G::HWH + lane + 1;
            const float2* t1 = t0 + HPL;
            const float bu = cls == 0 ? b_row<0, G::HWH>(q, t0, t1, std::make_integer_sequence<int, 25>{})
                                      : b_row<1, G::HWH>(q, t0, t1, std::make_integer_sequence<int, 25>{});
            const int k = vj * (n + 1) + vi;
            d = sigma * __ldg(sinv + k) * (bu - __ldg(g + k));
        } else if (!fast && vi >= 0 && vj >= 0 && vi <= n && vj <= n) {
            const HL vhx{sH, HPL, i0 - 2, 2 * (j0 - 2), false};
            const HL vhy{sH, HPL, i0 - 2, 2 * (j0 - 2), true};
            const SVert<float, G::PW> vp{sP, i0 - 3, j0 - 3};
            Acc<float> a;
            cell_apply_auto<false, false, true, false, false>(vi, vj, n, c, vhx, vhy, vp, a);
            const int k = vj * (n + 1) + vi;
            d = sigma * __ldg(sinv + k) * (a.bu - __ldg(g + k));
        }
        sD[r * G::DW + lane] = d;
    }
    __syncthreads();

    // ---- new (u, p) on the owned cells (i0 + lane, j0 + r), lane < TX
    for (int r = warp; r < TY; r += NW) {
        if (lane >= TX) break;
        const int ci = i0 + lane, cj = j0 + r;
        if (ci > n || cj > n) continue;
        float2 o[4];
        if (fast) {
            float2 bt[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) bt[s] = f2(0.f, 0.f);
            const int bd = (r + 1) * G::DW + lane + 1;
            if (cls == 0) bt_rows<0, G::DW>(q, sD, bd, bt, std::make_integer_sequence<int, 9>{});
            else bt_rows<1, G::DW>(q, sD, bd, bt, std::make_integer_sequence<int, 9>{});
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float2 hc = sH[(s & 1) * HPL + (2 * (r + 2) + (s >> 1)) * G::HWH + lane + 2];
                const float ti = -q.TI[cls][s];
                o[s] = __ffma2_rn(f2(ti, ti), bt[s], hc);
            }
            if (inner) {
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int k = (2 * cj + (s >> 1)) * ld + 2 * ci + (s & 1);
                    u_out[k] = o[s].x;
                    u_out[n2 + k] = o[s].y;
                }
            } else {
                const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    if (!slot_exists(cn, s)) continue;
                    const int k = (2 * cj + (s >> 1)) * ld + 2 * ci + (s & 1);
                    const bool uk = slot_unknown(cn, s);
                    u_out[k] = uk ? o[s].x : 0.f;
                    u_out[n2 + k] = uk ? o[s].y : 0.f;
                }
            }
        } else {
            const HL vhx{sH, HPL, i0 - 2, 2 * (j0 - 2), false};
            const HL vhy{sH, HPL, i0 - 2, 2 * (j0 - 2), true};
            const SVert<float, G::DW> vd{sD, i0 - 1, j0 - 1};
            Acc<float> a;
            cell_apply_auto<false, true, false, true, false>(ci, cj, n, c, vhx, vhy, vd, a);
            const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!slot_exists(cn, s)) continue;
                const int k = (2 * cj + (s >> 1)) * ld + 2 * ci + (s & 1);
                float ox = 0.f, oy = 0.f;
                if (slot_unknown(cn, s)) {
                    const float w = tau * a.idg[s];
                    ox = vhx.at(ci, cj, s & 1, s >> 1) - w * a.bt[0][s];
                    oy = vhy.at(ci, cj, s & 1, s >> 1) - w * a.bt[1][s];
                }
                u_out[k] = ox;
                u_out[n2 + k] = oy;
            }
        }
        p_out[cj * (n + 1) + ci] = sP[(r + 3) * G::PW + lane + 3] + sD[(r + 1) * G::DW + lane + 1];
    }
    pdl_trigger();
}

template <int NW>
static cudaError_t pair_smem_attr() {
    return cudaFuncSetAttribute(k_uzawa_pair<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PairTile::bytes(kPairMaxRows));
}

cudaError_t prepare_uzawa_pair() {
    cudaError_t e = pair_smem_attr<8>();
    if (e == cudaSuccess) e = pair_smem_attr<4>();
    if (e == cudaSuccess) e = pair_smem_attr<12>();
    return e;
}

// Rows per tile for level size n: the least work on the busiest SM, (tiles per SM, rounded up) x
// (work of one tile, about ty + 4 rows of the u^{m-1/2} region), among the tile heights that keep
// at least two CTAs resident per SM.
template <int NW>
static int pair_rows(int n) {
    static int cache[3][32] = {};
    const int lv = 31 - __builtin_clz((unsigned)n);
    int& r = cache[NW > 8 ? 2 : NW > 4 ? 1 : 0][lv & 31];
    if (r) return r;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::max(sms, 1);
    const int cols = (n + 1 + PairTile::TX - 1) / PairTile::TX;
    double best = 1e300;
    int best_ty = 16;
    for (int ty = 8; ty <= kPairMaxRows; ++ty) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_uzawa_pair<NW>, 32 * NW, PairTile::bytes(ty)) !=
                cudaSuccess || per_sm < 2)
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

// rows = 0: chosen by pair_rows; otherwise fixed (rows + 4 = NW puts one row of the u^{m-1/2}
// region on each warp: the shortest CTA, for the small, latency-bound levels)
template <int NW>
static void launch_pair_v(cudaStream_t s, int n, int rows, const OpCoef<float>& c, float tau, float sigma,
                          const float* u, const float* p, const float* f, const float* g, const float* sinv,
                          float* u_out, float* p_out) {
    const int ty = rows > 0 ? rows : pair_rows<NW>(n);
    TileOrder ord;
    ord.cols = (n + 1 + PairTile::TX - 1) / PairTile::TX;
    ord.rows = (n + 1 + ty - 1) / ty;
    mid_band(n / 2, PairTile::TX, ord.cols, ord.c0, ord.nc);
    mid_band(n / 2, ty, ord.rows, ord.r0, ord.nr);
    const dim3 grid(ord.cols * ord.rows), blk(32 * NW);
    launch_pdl(k_uzawa_pair<NW>, grid, blk, PairTile::bytes(ty), s, n, ty, ord, c, make_pair_coef(c, tau), tau,
               sigma, u, p, f, g, sinv, u_out, p_out);
}

void launch_uzawa_pair(int variant, cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma,
                       const float* u, const float* p, const float* f, const float* g, const float* sinv,
                       float* u_out, float* p_out) {
    if (variant == 0) launch_pair_v<8>(s, n, 0, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
    else if (variant == 1) launch_pair_v<4>(s, n, 0, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
    else launch_pair_v<12>(s, n, 8, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
}

}  // namespace smg
