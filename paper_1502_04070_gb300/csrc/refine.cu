// refine.cu -- the float64 side of mixed-precision iterative refinement.
//
// Each refinement step solves A e = r approximately with float32 cycles and then updates
//     x <- x + e,     r <- r - A e
// in float64 storage.  GB300 has few float64 units, so A e is formed from float32 operations
// that lose nothing: the float32 correction e is exact, every float64 coefficient is split as
// c = c_hi + c_lo (two floats), the product c_hi * e is made exact with an FMA (TwoProduct), and
// the products are summed with TwoSum into a (hi, lo) pair, which is accurate to about 2^-48
// relative to sum |c| |e|.  Because e shrinks with the residual, the accumulated error of the
// updated residual stays far below the refinement tolerance; the solver still recomputes the true
// float64 residual before it reports convergence.
//
// GB300 also runs conversions and additions in float64 on its narrow float64 pipe, so during the
// refinement loop the residual r is kept as an unevaluated sum of two floats (hi + lo, about 48
// significant bits) in the float64 array's own 8-byte slots; per unknown the loop issues only the
// two float64 instructions of x += e.  x itself stays float64: its precision bounds the attainable
// residual, and with two floats the solve stalled at 1.8e-8 relative residual for beta = 1e8 on
// h = 1/512, where |A| |x| is large against |F|.
#include "cellops.cuh"
#include "kernels.cuh"

namespace smg {

struct DF {
    float hi, lo;
};

// s += (chi + clo) * v ; the intrinsics keep the compiler from fusing the exact steps
__device__ __forceinline__ void df_fma(DF& s, float chi, float clo, float v) {
    const float p = __fmul_rn(chi, v);
    const float pe = fmaf(chi, v, -p);            // chi * v = p + pe exactly
    const float t = __fadd_rn(s.hi, p);           // TwoSum(s.hi, p)
    const float bb = __fsub_rn(t, s.hi);
    const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s.hi = t;
    s.lo += e + pe + clo * v;
}

__device__ __forceinline__ double df_value(const DF& s) { return (double)s.hi + (double)s.lo; }

struct DFAcc {
    DF au[2][4];
    DF bu;
};

template <int O, int SQ, int R>
__device__ __forceinline__ void sq_rows_df(const OpCoef<float>& h, const OpCoef<float>& l, const float (&vx)[9],
                                           const float (&vy)[9], const float (&pq)[4], DFAcc& a) {
    if constexpr (R < sq_nrows(SQ)) {
        constexpr int L = sq_row(SQ, R), s = sq_slot(SQ, R);
#pragma unroll
        for (int m = 0; m < 9; ++m)
            if (couple(O, L, m)) {
                df_fma(a.au[0][s], h.A[O][L][m], l.A[O][L][m], vx[m]);
                df_fma(a.au[1][s], h.A[O][L][m], l.A[O][L][m], vy[m]);
            }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (couple(O, corner_node(q), L)) {
                df_fma(a.au[0][s], h.Bx[O][q][L], l.Bx[O][q][L], pq[q]);
                df_fma(a.au[1][s], h.By[O][q][L], l.By[O][q][L], pq[q]);
            }
        sq_rows_df<O, SQ, R + 1>(h, l, vx, vy, pq, a);
    }
}

template <int O, int SQ>
__device__ __forceinline__ void sq_b_df(const OpCoef<float>& h, const OpCoef<float>& l, const float (&vx)[9],
                                        const float (&vy)[9], DFAcc& a) {
#pragma unroll
    for (int m = 0; m < 9; ++m)
        if (couple(O, corner_node(SQ), m)) {
            df_fma(a.bu, h.Bx[O][SQ][m], l.Bx[O][SQ][m], vx[m]);
            df_fma(a.bu, h.By[O][SQ][m], l.By[O][SQ][m], vy[m]);
        }
}

// PL: the float32 correction e is in the planar layout (common.cuh)
template <int SQ, bool PL>
__device__ __forceinline__ void visit_df(int i, int j, int n, const OpCoef<float>& h, const OpCoef<float>& l,
                                         const float* __restrict__ eu, const float* __restrict__ ep, DFAcc& a) {
    const int si = i - (SQ & 1), sj = j - (SQ >> 1);
    if (si < 0 || sj < 0 || si >= n || sj >= n) return;
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    float vx[9], vy[9], pq[4];
    if constexpr (PL) {
        load_sq<true>(gviewp<false>(eu, n, 0), n, si, sj, vx);
        load_sq<true>(gviewp<false>(eu, n, 1), n, si, sj, vy);
        load_sq_p(gview(ep, pl_vpitch(n)), si, sj, pq);
    } else {
        load_sq<true>(gview(eu, 2 * n + 1), n, si, sj, vx);
        load_sq<true>(gview(eu + n2, 2 * n + 1), n, si, sj, vy);
        load_sq_p(gview(ep, n + 1), si, sj, pq);
    }
    if (orient(si, sj, n)) {
        sq_rows_df<1, SQ, 0>(h, l, vx, vy, pq, a);
        sq_b_df<1, SQ>(h, l, vx, vy, a);
    } else {
        sq_rows_df<0, SQ, 0>(h, l, vx, vy, pq, a);
        sq_b_df<0, SQ>(h, l, vx, vy, a);
    }
}

// The same rows from the merged stencils of class C (blocks off the mid-lines and at least two
// cells inside the boundary: every window lies inside the arrays, every term is decided at compile
// time), with the x and y components side by side in packed FP32x2 instructions: the velocity
// block applies one coefficient to (e_x, e_y), B^T an (x, y) coefficient pair to (p, p), and B an
// (x, y) pair to (e_x, e_y) whose two halves are summed at the end.  Each lane of every packed
// instruction is a correctly rounded float operation, so TwoProduct and TwoSum stay exact.
struct DFPairCoef {   // split float64 coefficients (hi + lo) as (x, y) pairs, classes 0 and 1
    float2 MAh[2][4][25], MAl[2][4][25];
    float2 MBTh[2][4][9], MBTl[2][4][9];
    float2 MBh[2][25], MBl[2][25];
};

static DFPairCoef make_df_pairs(const OpCoef<float>& h, const OpCoef<float>& l) {
    DFPairCoef q{};
    for (int k = 0; k < 2; ++k) {
        for (int s = 0; s < 4; ++s) {
            for (int w = 0; w < 25; ++w) {
                q.MAh[k][s][w] = make_float2(h.MA[k][s][w], h.MA[k][s][w]);
                q.MAl[k][s][w] = make_float2(l.MA[k][s][w], l.MA[k][s][w]);
            }
            for (int v = 0; v < 9; ++v) {
                q.MBTh[k][s][v] = make_float2(h.MBTx[k][s][v], h.MBTy[k][s][v]);
                q.MBTl[k][s][v] = make_float2(l.MBTx[k][s][v], l.MBTy[k][s][v]);
            }
        }
        for (int w = 0; w < 25; ++w) {
            q.MBh[k][w] = make_float2(h.MBx[k][w], h.MBy[k][w]);
            q.MBl[k][w] = make_float2(l.MBx[k][w], l.MBy[k][w]);
        }
    }
    return q;
}

struct DF2 {
    float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// s += (chi + clo) * v on both lanes (TwoProduct of chi * v, TwoSum into s.hi)
__device__ __forceinline__ void df2_fma(DF2& s, float2 chi, float2 clo, float2 v) {
    const float2 p = __fmul2_rn(chi, v);
    const float2 pe = __ffma2_rn(chi, v, neg2(p));
    const float2 t = __fadd2_rn(s.hi, p);
    const float2 bb = __fadd2_rn(t, neg2(s.hi));
    const float2 e = __fadd2_rn(__fadd2_rn(s.hi, neg2(__fadd2_rn(t, neg2(bb)))), __fadd2_rn(p, neg2(bb)));
    s.hi = t;
    s.lo = __fadd2_rn(s.lo, __fadd2_rn(e, __ffma2_rn(clo, v, pe)));
}

template <int C, int S, int K>
__device__ __forceinline__ void ma_df2(const DFPairCoef& q, float2 v, DF2 (&au)[4]) {
    if constexpr (nz_MA(C, S, K)) df2_fma(au[S], q.MAh[C][S][K], q.MAl[C][S][K], v);
}
template <int C, int K>
__device__ __forceinline__ void win_df2(const DFPairCoef& q, const float (&wx)[25], const float (&wy)[25],
                                        DF2 (&au)[4], DF2& bu) {
    if constexpr (need_win(C, true, true, K)) {
        const float2 v = make_float2(wx[K], wy[K]);
        ma_df2<C, 0, K>(q, v, au);
        ma_df2<C, 1, K>(q, v, au);
        ma_df2<C, 2, K>(q, v, au);
        ma_df2<C, 3, K>(q, v, au);
        if constexpr (nz_MB(C, K)) df2_fma(bu, q.MBh[C][K], q.MBl[C][K], v);
    }
}
template <int C, int S, int V>
__device__ __forceinline__ void mbt_df2(const DFPairCoef& q, float2 pv, DF2 (&au)[4]) {
    if constexpr (nz_MBT(C, S, V)) df2_fma(au[S], q.MBTh[C][S][V], q.MBTl[C][S][V], pv);
}
template <int C, int V>
__device__ __forceinline__ void vwin_df2(const DFPairCoef& q, const float (&pw)[9], DF2 (&au)[4]) {
    if constexpr (need_vwin(C, V)) {
        const float2 pv = make_float2(pw[V], pw[V]);
        mbt_df2<C, 0, V>(q, pv, au);
        mbt_df2<C, 1, V>(q, pv, au);
        mbt_df2<C, 2, V>(q, pv, au);
        mbt_df2<C, 3, V>(q, pv, au);
    }
}
// CHECKED: blocks at the boundary (off the mid-lines) read with range tests and the Dirichlet mask
// Window point W of cell (i, j) from a planar float32 velocity array (both components in one 8-byte
// load; every window point inside the arrays)
template <int C, int W>
__device__ __forceinline__ void win_pair1(int i, int j, const float* __restrict__ eu, int rs, int ps, float (&wx)[25],
                                          float (&wy)[25]) {
    if constexpr (need_win(C, true, true, W)) {
        constexpr int dx = W % 5 - 2, dy = W / 5 - 2;
        const float2 v = __ldg(reinterpret_cast<const float2*>(eu + (dx & 1) * ps + (2 * j + dy) * rs +
                                                               2 * (i + (dx >> 1))));
        wx[W] = v.x;
        wy[W] = v.y;
    }
}
template <int C, int... W>
__device__ __forceinline__ void win_pairs(int i, int j, int n, const float* __restrict__ eu, float (&wx)[25],
                                          float (&wy)[25], std::integer_sequence<int, W...>) {
    const int rs = 2 * pl_pitch(n), ps = rs * pl_rows(n);
    (win_pair1<C, W>(i, j, eu, rs, ps, wx, wy), ...);
}

template <int C, bool CHECKED, bool PL, int... K, int... V>
__device__ __forceinline__ void merged_df(int i, int j, int n, const DFPairCoef& q, const float* __restrict__ eu,
                                          const float* __restrict__ ep, DFAcc& a, std::integer_sequence<int, K...>,
                                          std::integer_sequence<int, V...>) {
    const int n2 = (2 * n + 1) * (2 * n + 1);
    float wx[25], wy[25], pw[9];
    if constexpr (PL && CHECKED) {
        win_load<C, true, true, true>(i, j, n, gviewp<false>(eu, n, 0), gviewp<false>(eu, n, 1), wx, wy,
                                      std::make_integer_sequence<int, 25>{});
        vwin_load<C>(i, j, n, gview(ep, pl_vpitch(n)), pw, std::make_integer_sequence<int, 9>{});
    } else if constexpr (PL) {
        win_pairs<C>(i, j, n, eu, wx, wy, std::make_integer_sequence<int, 25>{});
        vwin_load<C>(i, j, n, gviewu(ep, pl_vpitch(n)), pw, std::make_integer_sequence<int, 9>{});
    } else if constexpr (CHECKED) {
        win_load<C, true, true, true>(i, j, n, gview(eu, 2 * n + 1), gview(eu + n2, 2 * n + 1), wx, wy,
                                      std::make_integer_sequence<int, 25>{});
        vwin_load<C>(i, j, n, gview(ep, n + 1), pw, std::make_integer_sequence<int, 9>{});
    } else {
        win_load<C, true, true, false>(i, j, n, gviewu(eu, 2 * n + 1), gviewu(eu + n2, 2 * n + 1), wx, wy,
                                       std::make_integer_sequence<int, 25>{});
        vwin_load<C>(i, j, n, gviewu(ep, n + 1), pw, std::make_integer_sequence<int, 9>{});
    }
    DF2 au[4], bu;
#pragma unroll
    for (int s = 0; s < 4; ++s) au[s] = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    bu = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    (win_df2<C, K>(q, wx, wy, au, bu), ...);
    (vwin_df2<C, V>(q, pw, au), ...);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a.au[0][s] = DF{au[s].hi.x, au[s].lo.x};
        a.au[1][s] = DF{au[s].hi.y, au[s].lo.y};
    }
    // B row: the x and y halves summed (TwoSum of the high parts)
    const float t = __fadd_rn(bu.hi.x, bu.hi.y);
    const float bb = __fsub_rn(t, bu.hi.x);
    const float e = __fadd_rn(__fsub_rn(bu.hi.x, __fsub_rn(t, bb)), __fsub_rn(bu.hi.y, bb));
    a.bu = DF{t, __fadd_rn(__fadd_rn(bu.lo.x, bu.lo.y), e)};
}

// ---------------------------------------------------------------------------------------------
// two-float ("double-float") state

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ float2 renorm(float s, float e) {
    const float hi = __fadd_rn(s, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}
// a - (b.hi + b.lo)
__device__ __forceinline__ float2 df_sub(float2 a, const DF& b) {
    float s, e;
    two_sum(a.x, -b.hi, s, e);
    return renorm(s, __fadd_rn(e, __fsub_rn(a.y, b.lo)));
}

template <bool PL>
__global__ void __launch_bounds__(NT, 4) k_ir_update_df(int n, const __grid_constant__ OpCoef<float> ch,
                                                     const __grid_constant__ OpCoef<float> cl,
                                                     const __grid_constant__ DFPairCoef cq,
                                                     const float* __restrict__ eu, const float* __restrict__ ep,
                                                     double* __restrict__ xu, double* __restrict__ xp,
                                                     float2* __restrict__ ru, float2* __restrict__ rp,
                                                     float* __restrict__ r32u, float* __restrict__ r32p,
                                                     double* __restrict__ partial, double* __restrict__ wpartial,
                                                     double wscale, int dom) {
    pdl_wait();
    CELL_INDEX
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    float ss = 0.f;
    // (triangles at vertex i) x_p,i of the updated pressure; times wscale = h^2 / 6 per block, the
    // zero-mean projection's numerator sum_i w_i x_p,i (float64 work kept to the additions)
    double wp = 0.0;
    if (active) {
        DFAcc a;
#pragma unroll
        for (int s = 0; s < 4; ++s) a.au[0][s] = a.au[1][s] = DF{0.f, 0.f};
        a.bu = DF{0.f, 0.f};
        const int hh = n >> 1, bi0 = blockIdx.x * blockDim.x, bj0 = blockIdx.y * blockDim.y;
        const bool single = (hh < bi0 || hh >= bi0 + (int)blockDim.x) && (hh < bj0 || hh >= bj0 + (int)blockDim.y);
        constexpr auto K25 = std::make_integer_sequence<int, 25>{};
        constexpr auto V9 = std::make_integer_sequence<int, 9>{};
        if (single && block_interior(n, 2)) {
            if (orient(bi0, bj0, n) == 0) merged_df<0, false, PL>(i, j, n, cq, eu, ep, a, K25, V9);
            else merged_df<1, false, PL>(i, j, n, cq, eu, ep, a, K25, V9);
        } else if (single) {
            if (orient(bi0, bj0, n) == 0) merged_df<0, true, PL>(i, j, n, cq, eu, ep, a, K25, V9);
            else merged_df<1, true, PL>(i, j, n, cq, eu, ep, a, K25, V9);
        } else {
            visit_df<0, PL>(i, j, n, ch, cl, eu, ep, a);
            visit_df<1, PL>(i, j, n, ch, cl, eu, ep, a);
            visit_df<2, PL>(i, j, n, ch, cl, eu, ep, a);
            visit_df<3, PL>(i, j, n, ch, cl, eu, ep, a);
        }
        const CellNodes cn = cell_nodes_dom(i, j, n, dom);
        const int ld = 2 * n + 1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_unknown(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const size_t idx = (size_t)Y * ld + X;
            const size_t i32 = PL ? (size_t)pl_u(n, X, Y) : idx;   // the float32 arrays' index
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
                const size_t k = comp * n2 + idx, k32 = PL ? i32 + comp : k;
                xu[k] += (double)eu[k32];
                const float2 r = df_sub(ru[k], a.au[comp][s]);
                ru[k] = r;
                r32u[k32] = r.x;
                ss = fmaf(r.x, r.x, ss);
            }
        }
        const size_t vi = (size_t)j * (n + 1) + i, vi32 = PL ? (size_t)j * pl_vpitch(n) + i : vi;
        if (!(dom == kDomL && l_masked_vertex(i, j, n))) {   // vertices outside the L keep zero
            const double xpn = xp[vi] + (double)ep[vi32];
            xp[vi] = xpn;
            wp = (double)vertex_triangles_dom(i, j, n, dom) * xpn;
            const float2 r = df_sub(rp[vi], a.bu);
            rp[vi] = r;
            r32p[vi32] = r.x;
            ss = fmaf(r.x, r.x, ss);
        }
    }
    const double2 t = block_sum2_fd(ss, wp, tid);
    if (tid == 0) {
        partial[blockIdx.y * gridDim.x + blockIdx.x] = t.x;
        wpartial[blockIdx.y * gridDim.x + blockIdx.x] = t.y * wscale;
    }
    pdl_trigger();
}

// true float64 residual r = F - A x (x, F float64), written as two-float r and float32 r32 (PL: r32
// in the planar layout)
template <bool PL>
__global__ void __launch_bounds__(NT) k_residual_df(int n, const __grid_constant__ OpCoef<double> c,
                                                    const double* __restrict__ u, const double* __restrict__ p,
                                                    const double* __restrict__ f, const double* __restrict__ g,
                                                    float2* __restrict__ ru, float2* __restrict__ rp,
                                                    float* __restrict__ r32u, float* __restrict__ r32p,
                                                    double* __restrict__ partial, int dom) {
    pdl_wait();
    CELL_INDEX
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    double ss = 0.0;
    if (active) {
        Acc<double> a;
        cell_apply_auto<true, true, true, false, true>(i, j, n, c, gview(u, 2 * n + 1), gview(u + n2, 2 * n + 1),
                                                  gview(p, n + 1), a);
        const CellNodes cn = cell_nodes_dom(i, j, n, dom);
        const int ld = 2 * n + 1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const size_t idx = (size_t)Y * ld + X;
            const size_t i32 = PL ? (size_t)pl_u(n, X, Y) : idx;
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
                const size_t k = comp * n2 + idx;
                double r = 0.0;
                if (slot_unknown(cn, s)) r = f[k] - a.au[comp][s] - a.bt[comp][s];
                const float hi = (float)r;
                ru[k] = make_float2(hi, (float)(r - (double)hi));
                r32u[PL ? i32 + comp : k] = hi;
                ss += r * r;
            }
        }
        const size_t vi = (size_t)j * (n + 1) + i;
        const double r = (dom == kDomL && l_masked_vertex(i, j, n)) ? 0.0 : g[vi] - a.bu;
        const float hi = (float)r;
        rp[vi] = make_float2(hi, (float)(r - (double)hi));
        r32p[PL ? (size_t)j * pl_vpitch(n) + i : vi] = hi;
        ss += r * r;
    }
    const double t = block_sum2d(ss, tid);
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
    pdl_trigger();
}

void launch_ir_update_df(cudaStream_t s, int n, const OpCoef<float>& chi, const OpCoef<float>& clo,
                         const float* eu, const float* ep, double* xu, double* xp, double* ru, double* rp,
                         float* r32u, float* r32p, double* partial, double* wpartial, bool planar, int dom) {
    launch_pdl(planar ? k_ir_update_df<true> : k_ir_update_df<false>, cells_grid(n), dim3(BX, BY), 0, s, n, chi, clo,
               make_df_pairs(chi, clo), eu, ep, xu, xp, reinterpret_cast<float2*>(ru), reinterpret_cast<float2*>(rp), r32u,
               r32p, partial, wpartial, 1.0 / (6.0 * (double)n * (double)n), dom);
}

void launch_residual_df(cudaStream_t s, int n, const OpCoef<double>& c, const double* u, const double* p,
                        const double* f, const double* g, double* ru, double* rp, float* r32u, float* r32p,
                        double* partial, bool planar, int dom) {
    launch_pdl(planar ? k_residual_df<true> : k_residual_df<false>, cells_grid(n), dim3(BX, BY), 0, s, n, c, u, p, f,
               g, reinterpret_cast<float2*>(ru), reinterpret_cast<float2*>(rp), r32u, r32p, partial, dom);
}

}  // namespace smg
