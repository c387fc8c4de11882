// kernels.cu -- matrix-free kernels of the coupled multigrid cycle (Secs. 3-5).
//
// Every kernel runs one thread per cell (i, j) of a level, i, j in [0, N] (see common.cuh for the
// owned nodes and the square-local matrices).  The operator rows are the merged node stencils of
// the cell's stencil class (the orientations of its four squares; warp-uniform except where a warp
// meets one of the mid-lines x = 1/2, y = 1/2), with structurally-zero entries removed at compile
// time.  Blocks whose cells all lie at least two cells inside the boundary read without any test.
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "cellops.cuh"
#include "kernels.cuh"

namespace smg {

int cells_blocks(int n) { return ((n + 1 + BX - 1) / BX) * ((n + 1 + BY - 1) / BY); }

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("STOKES_MG_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

bool fuse_prolong_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("STOKES_MG_FUSE_PROLONG");
        return !(e && e[0] == '0');
    }();
    return on;
}

__constant__ double c_W2d[2][9][5][5];
__constant__ float c_W2f[2][9][5][5];

template <typename T> __device__ __forceinline__ T W2(int o, int L, int fb, int fa);
template <> __device__ __forceinline__ double W2<double>(int o, int L, int fb, int fa) { return c_W2d[o][L][fb][fa]; }
template <> __device__ __forceinline__ float W2<float>(int o, int L, int fb, int fa) { return c_W2f[o][L][fb][fa]; }

cudaError_t upload_transfer_weights(const double* P2) {
    float tmp[2 * 9 * 25];
    for (int i = 0; i < 2 * 9 * 25; ++i) tmp[i] = (float)P2[i];
    cudaError_t e = cudaMemcpyToSymbol(c_W2d, P2, sizeof(double) * 2 * 9 * 25);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_W2f, tmp, sizeof(float) * 2 * 9 * 25);
}

// ------------------------------------------------------------------------------------------
// r = F - A x  (eq. gen:bil:mv), optional sum of squares.  PL: float32 arrays in the planar layout
// (common.cuh; then ru2, rp2 are null).
template <typename T, typename TO, bool PL>
__global__ void __launch_bounds__(NT) k_residual(int n, const __grid_constant__ OpCoef<T> c,
                                                 const T* __restrict__ u, const T* __restrict__ p,
                                                 const T* __restrict__ f, const T* __restrict__ g,
                                                 TO* __restrict__ ru, TO* __restrict__ rp,
                                                 double* __restrict__ partial, float* __restrict__ ru2,
                                                 float* __restrict__ rp2, int dom) {
    static_assert(!PL || (sizeof(T) == 4 && sizeof(TO) == 4), "the planar layout is float32 only");
    pdl_wait();
    CELL_INDEX
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    const int vld = PL ? pl_vpitch(n) : n + 1;
    double ss = 0.0;
    if (active) {
        Acc<T> a;
        if constexpr (PL) {
            if (block_interior(n, 2))
                cell_apply_auto<true, true, true, false, false>(i, j, n, c, gviewp<true>(u, n, 0), gviewp<true>(u, n, 1),
                                                                gviewu(p, vld), a);
            else
                cell_apply_auto<true, true, true, false, true>(i, j, n, c, gviewp<false>(u, n, 0), gviewp<false>(u, n, 1),
                                                               gview(p, vld), a);
        } else {
            if (block_interior(n, 2))
                cell_apply_auto<true, true, true, false, false>(i, j, n, c, gviewu(u, 2 * n + 1),
                                                                gviewu(u + n2, 2 * n + 1), gviewu(p, n + 1), a);
            else
                cell_apply_auto<true, true, true, false, true>(i, j, n, c, gview(u, 2 * n + 1), gview(u + n2, 2 * n + 1),
                                                               gview(p, n + 1), a);
        }
        const CellNodes cn = cell_nodes_dom(i, j, n, dom);
        const int ld = 2 * n + 1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const size_t idx = PL ? (size_t)pl_u(n, X, Y) : (size_t)Y * ld + X;
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
                const size_t k = PL ? idx + comp : comp * n2 + idx;
                TO r = TO(0);
                if (slot_unknown(cn, s)) {
                    const T rr = f[k] - a.au[comp][s] - a.bt[comp][s];
                    r = (TO)rr;
                    ss += (double)rr * (double)rr;
                }
                ru[k] = r;
                if (!PL && ru2) ru2[k] = (float)r;
            }
        }
        const size_t vi = (size_t)j * vld + i;
        const T r = (dom == kDomL && l_masked_vertex(i, j, n)) ? T(0) : g[vi] - a.bu;
        rp[vi] = (TO)r;
        if (!PL && rp2) rp2[vi] = (float)r;
        ss += (double)r * (double)r;
    }
    if (partial) {
        const double t = block_sum2d(ss, tid);
        if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
    pdl_trigger();
}

// float32: four CTAs per SM (64 registers; a few spilled) for more loads in flight
template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 4 : 1) k_uzawa_u(int n, const __grid_constant__ OpCoef<T> c, T tau,
                                                const T* __restrict__ u, const T* __restrict__ p,
                                                const T* __restrict__ f, T* __restrict__ uh, int dom) {
    pdl_wait();
    CELL_INDEX
    if (!active) return;
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    Acc<T> a;
    if (block_interior(n, 2))
        cell_apply_auto<true, true, false, true, false>(i, j, n, c, gviewu(u, 2 * n + 1), gviewu(u + n2, 2 * n + 1),
                                                        gviewu(p, n + 1), a);
    else
        cell_apply_auto<true, true, false, true, true>(i, j, n, c, gview(u, 2 * n + 1), gview(u + n2, 2 * n + 1),
                                                       gview(p, n + 1), a);
    const CellNodes cn = cell_nodes_dom(i, j, n, dom);
    const int ld = 2 * n + 1;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (!slot_exists(cn, s)) continue;
        int X, Y;
        slot_pos(i, j, s, X, Y);
        const size_t idx = (size_t)Y * ld + X;
        const bool unk = slot_unknown(cn, s);
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
            const size_t k = comp * n2 + idx;
            uh[k] = unk ? u[k] + tau * (f[k] - a.au[comp][s] - a.bt[comp][s]) * a.idg[s] : T(0);
        }
    }
    pdl_trigger();
}

template <typename T>
__global__ void __launch_bounds__(NT) k_uzawa_p(int n, const __grid_constant__ OpCoef<T> c, T sigma,
                                                const T* __restrict__ uh, T* __restrict__ p,
                                                const T* __restrict__ g, const T* __restrict__ sinv,
                                                T* __restrict__ dp) {
    pdl_wait();
    CELL_INDEX
    if (!active) return;
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    Acc<T> a;
    if (block_interior(n, 1))
        cell_apply_auto<false, false, true, false, false>(i, j, n, c, gviewu(uh, 2 * n + 1), gviewu(uh + n2, 2 * n + 1),
                                                          gviewu((const T*)nullptr, n + 1), a);
    else
        cell_apply_auto<false, false, true, false, false>(i, j, n, c, gview(uh, 2 * n + 1), gview(uh + n2, 2 * n + 1),
                                                          gview((const T*)nullptr, n + 1), a);
    const size_t vi = (size_t)j * (n + 1) + i;
    // p^{m} = p^{m-1} - sigma Shat^{-1} (g - B u^{m-1/2})
    const T d = sigma * sinv[vi] * (a.bu - g[vi]);
    p[vi] += d;
    dp[vi] = d;
    pdl_trigger();
}

template <typename T>
__global__ void __launch_bounds__(NT) k_uzawa_u2(int n, const __grid_constant__ OpCoef<T> c, T tau,
                                                 const T* __restrict__ uh, const T* __restrict__ dp,
                                                 T* __restrict__ u, int dom) {
    pdl_wait();
    CELL_INDEX
    if (!active) return;
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    Acc<T> a;
    if (block_interior(n, 1))
        cell_apply_auto<false, true, false, true, false>(i, j, n, c, gviewu((const T*)nullptr, 2 * n + 1),
                                                         gviewu((const T*)nullptr, 2 * n + 1), gviewu(dp, n + 1), a);
    else
        cell_apply_auto<false, true, false, true, false>(i, j, n, c, gview((const T*)nullptr, 2 * n + 1),
                                                         gview((const T*)nullptr, 2 * n + 1), gview(dp, n + 1), a);
    const CellNodes cn = cell_nodes_dom(i, j, n, dom);
    const int ld = 2 * n + 1;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (!slot_exists(cn, s)) continue;
        int X, Y;
        slot_pos(i, j, s, X, Y);
        const size_t idx = (size_t)Y * ld + X;
        const bool unk = slot_unknown(cn, s);
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
            const size_t k = comp * n2 + idx;
            // u^{m} = u^{m-1/2} - tau Ahat^{-1} B^T (p^{m} - p^{m-1})
            u[k] = unk ? uh[k] - tau * a.bt[comp][s] * a.idg[s] : T(0);
        }
    }
    pdl_trigger();
}

template <typename T>
void launch_uzawa(cudaStream_t s, int n, const OpCoef<T>& c, T tau, T sigma, T* u, T* p, const T* f,
                  const T* g, const T* sinv, T* uh, T* dp, int bx, int by, int dom) {
    const dim3 blk(bx, by), grid((n + 1 + bx - 1) / bx, (n + 1 + by - 1) / by);
    launch_pdl(k_uzawa_u<T>, grid, blk, 0, s, n, c, tau, u, p, f, uh, dom);
    // dp = 0 where Shat^{-1} = 0: on the L the vertices outside it
    launch_pdl(k_uzawa_p<T>, grid, blk, 0, s, n, c, sigma, uh, p, g, sinv, dp);
    launch_pdl(k_uzawa_u2<T>, grid, blk, 0, s, n, c, tau, uh, dp, u, dom);
}

// ------------------------------------------------------------------------------------------
// normal-equation smoother: z = L^{-1} r  then  x += tau L^{-1} A z
template <typename T>
__global__ void __launch_bounds__(NT) k_scale_L(int n, const __grid_constant__ OpCoef<T> c,
                                                T* __restrict__ zu, T* __restrict__ zp,
                                                const T* __restrict__ sinv) {
    pdl_wait();
    CELL_INDEX
    if (!active) return;
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    Acc<T> a;
    cell_apply_auto<false, false, false, true, false>(i, j, n, c, gview((const T*)nullptr, 2 * n + 1),
                                                 gview((const T*)nullptr, 2 * n + 1), gview((const T*)nullptr, n + 1), a);
    const CellNodes cn = cell_nodes(i, j, n);
    const int ld = 2 * n + 1;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (!slot_unknown(cn, s)) continue;
        int X, Y;
        slot_pos(i, j, s, X, Y);
        const size_t idx = (size_t)Y * ld + X;
        zu[idx] *= a.idg[s];
        zu[n2 + idx] *= a.idg[s];
    }
    const size_t vi = (size_t)j * (n + 1) + i;
    zp[vi] *= sinv[vi];
    pdl_trigger();
}

template <typename T>
__global__ void __launch_bounds__(NT) k_normal_update(int n, const __grid_constant__ OpCoef<T> c, T tau,
                                                      const T* __restrict__ zu, const T* __restrict__ zp,
                                                      const T* __restrict__ sinv, T* __restrict__ u,
                                                      T* __restrict__ p) {
    pdl_wait();
    CELL_INDEX
    if (!active) return;
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    Acc<T> a;
    cell_apply_auto<true, true, true, true, false>(i, j, n, c, gview(zu, 2 * n + 1), gview(zu + n2, 2 * n + 1), gview(zp, n + 1), a);
    const CellNodes cn = cell_nodes(i, j, n);
    const int ld = 2 * n + 1;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (!slot_unknown(cn, s)) continue;
        int X, Y;
        slot_pos(i, j, s, X, Y);
        const size_t idx = (size_t)Y * ld + X;
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) u[comp * n2 + idx] += tau * (a.au[comp][s] + a.bt[comp][s]) * a.idg[s];
    }
    const size_t vi = (size_t)j * (n + 1) + i;
    p[vi] += tau * sinv[vi] * a.bu;
    pdl_trigger();
}

template <typename T>
void launch_normal_eq(cudaStream_t s, int n, const OpCoef<T>& c, T tau, T* u, T* p, const T* f,
                      const T* g, const T* sinv, T* zu, T* zp) {
    const dim3 grid = cells_grid(n), blk(BX, BY);
    launch_pdl(k_residual<T, T, false>, grid, blk, 0, s, n, c, u, p, f, g, zu, zp, nullptr, nullptr, nullptr,
               (int)kDomSquare);
    launch_pdl(k_scale_L<T>, grid, blk, 0, s, n, c, zu, zp, sinv);
    launch_pdl(k_normal_update<T>, grid, blk, 0, s, n, c, tau, zu, zp, sinv, u, p);
}

template <typename T, typename TO>
void launch_residual(cudaStream_t s, int n, const OpCoef<T>& c, const T* u, const T* p, const T* f,
                     const T* g, TO* ru, TO* rp, double* partial, float* ru2, float* rp2, int dom) {
    launch_pdl(k_residual<T, TO, false>, cells_grid(n), dim3(BX, BY), 0, s, n, c, u, p, f, g, ru, rp, partial, ru2, rp2,
               dom);
}

void launch_residual_planar(cudaStream_t s, int n, const OpCoef<float>& c, const float* u, const float* p,
                            const float* f, const float* g, float* ru, float* rp) {
    launch_pdl(k_residual<float, float, true>, cells_grid(n), dim3(BX, BY), 0, s, n, c, u, p, f, g, ru, rp,
               (double*)nullptr, (float*)nullptr, (float*)nullptr, (int)kDomSquare);
}

// ------------------------------------------------------------------------------------------
// Restriction (Sec. 3): coarse value = sum over fine points of (coarse basis at the point) x r.
// Every fine point is owned by one coarse square (local fine offsets 0..3 in each direction);
// points on the far edges belong to the neighbouring square, where the weights of the nodes not
// shared with it vanish, so the sum over the 1-4 squares of a coarse node's patch is exact.
template <int O, int SQ, int R, typename T>
__device__ __forceinline__ void restrict_rows(const T (&v)[2][4][4], T (&acc)[2][4]) {
    if constexpr (R < sq_nrows(SQ)) {
        constexpr int L = sq_row(SQ, R), s = sq_slot(SQ, R);
#pragma unroll
        for (int fb = 0; fb < 4; ++fb)
#pragma unroll
            for (int fa = 0; fa < 4; ++fa) {
                const T w = W2<T>(O, L, fb, fa);
                acc[0][s] = fma(w, v[0][fb][fa], acc[0][s]);
                acc[1][s] = fma(w, v[1][fb][fa], acc[1][s]);
            }
        restrict_rows<O, SQ, R + 1>(v, acc);
    }
}

// global arrays go through the read-only path; shared-memory arrays (the coarse sub-cycle) do not
template <bool LDG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
    if constexpr (LDG) return __ldg(p);
    else return *p;
}

// Strides of the arrays a transfer reads and writes, each pointer at the array's (0, 0) entry:
// the dense level arrays (dense_layout), the padded shared-memory arrays of the coarse cycle, or
// float32 levels in the planar layout (template flags PF / PC of the fine / coarse level; there the
// row stride is in floats, the component stride is 1 and psf / psc is the parity-plane stride).
struct XferLayout {
    int ldf, n2f;   // fine velocity: row stride, component stride
    int ldpf;       // fine vertex array: row stride
    int ldc, n2c;   // coarse velocity
    int ldpc;       // coarse vertex array
    int psf = 0, psc = 0;
};
__host__ __device__ __forceinline__ XferLayout dense_layout(int nc) {
    const int ldf = 4 * nc + 1, ldc = 2 * nc + 1;
    return XferLayout{ldf, ldf * ldf, 2 * nc + 1, ldc, ldc * ldc, nc + 1};
}
__host__ __device__ __forceinline__ XferLayout xfer_layout(int nc, bool pf, bool pc) {
    XferLayout l = dense_layout(nc);
    if (pf) {
        const int nf = 2 * nc;
        l.ldf = 2 * pl_pitch(nf);
        l.n2f = 1;
        l.ldpf = pl_vpitch(nf);
        l.psf = l.ldf * pl_rows(nf);
    }
    if (pc) {
        l.ldc = 2 * pl_pitch(nc);
        l.n2c = 1;
        l.ldpc = pl_vpitch(nc);
        l.psc = l.ldc * pl_rows(nc);
    }
    return l;
}
// offset of lattice point (X, Y), component 0, in a velocity array of row stride ld (plane stride ps)
template <bool PLN>
__host__ __device__ __forceinline__ int lat_at(int X, int Y, int ld, int ps) {
    if constexpr (PLN) return (X & 1) * ps + Y * ld + (X >> 1) * 2;
    else return Y * ld + X;
}

template <int SQ, bool LDG, bool PF, typename T>
__device__ __forceinline__ void restrict_visit(int I, int J, int nc, const T* __restrict__ ru, T (&acc)[2][4],
                                               const XferLayout& lay) {
    const int SI = I - (SQ & 1), SJ = J - (SQ >> 1);
    if (SI < 0 || SJ < 0 || SI >= nc || SJ >= nc) return;
    T v[2][4][4];
#pragma unroll
    for (int fb = 0; fb < 4; ++fb)
#pragma unroll
        for (int fa = 0; fa < 4; ++fa) {
            const int k = lat_at<PF>(4 * SI + fa, 4 * SJ + fb, lay.ldf, lay.psf);
            v[0][fb][fa] = ldv<LDG>(ru + k);
            v[1][fb][fa] = ldv<LDG>(ru + lay.n2f + k);
        }
    if (orient(SI, SJ, nc)) restrict_rows<1, SQ, 0>(v, acc);
    else restrict_rows<0, SQ, 0>(v, acc);
}

// coarse cell (i, j) of level nc: its owned coarse velocity nodes and vertex
template <bool LDG, typename T, bool PF = false, bool PC = false>
__device__ __forceinline__ void restrict_cell(int i, int j, int nc, const T* __restrict__ ru, const T* __restrict__ rp,
                                              T* __restrict__ fc, T* __restrict__ gc, const XferLayout& lay,
                                              int dom = kDomSquare) {
    T acc[2][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[0][s] = acc[1][s] = T(0);
    restrict_visit<0, LDG, PF>(i, j, nc, ru, acc, lay);
    restrict_visit<1, LDG, PF>(i, j, nc, ru, acc, lay);
    restrict_visit<2, LDG, PF>(i, j, nc, ru, acc, lay);
    restrict_visit<3, LDG, PF>(i, j, nc, ru, acc, lay);
    const CellNodes cn = cell_nodes_dom(i, j, nc, dom);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (!slot_exists(cn, s)) continue;
        int X, Y;
        slot_pos(i, j, s, X, Y);
        const int k = lat_at<PC>(X, Y, lay.ldc, lay.psc);
        const bool unk = slot_unknown(cn, s);
        fc[k] = unk ? acc[0][s] : T(0);
        fc[lay.n2c + k] = unk ? acc[1][s] : T(0);
    }
    // P1: the coarse hat function is 1 at (2i, 2j), 1/2 at the fine vertices halfway along the
    // coarse edges through it (horizontal, vertical, and the diagonal of each square whose cut
    // passes through the vertex), 0 elsewhere.
    const int nf = 2 * nc, ldf = lay.ldpf;
    const int x = 2 * i, y = 2 * j;
    T s = rp[y * ldf + x];
    T half = T(0);
    if (x > 0) half += rp[y * ldf + x - 1];
    if (x < nf) half += rp[y * ldf + x + 1];
    if (y > 0) half += rp[(y - 1) * ldf + x];
    if (y < nf) half += rp[(y + 1) * ldf + x];
    // diagonal neighbours (dx, dy): square (i + min(dx,0), j + min(dy,0)); orientation 0 joins
    // (dx, dy) = (+,+) / (-,-), orientation 1 joins (+,-) / (-,+)
    if (x < nf && y < nf && orient(i, j, nc) == 0) half += rp[(y + 1) * ldf + x + 1];
    if (x > 0 && y > 0 && orient(i - 1, j - 1, nc) == 0) half += rp[(y - 1) * ldf + x - 1];
    if (x < nf && y > 0 && orient(i, j - 1, nc) == 1) half += rp[(y - 1) * ldf + x + 1];
    if (x > 0 && y < nf && orient(i - 1, j, nc) == 1) half += rp[(y + 1) * ldf + x - 1];
    gc[j * lay.ldpc + i] = (dom == kDomL && l_masked_vertex(i, j, nc)) ? T(0) : s + T(0.5) * half;
}

// With uc, pc given, the coarse iterate is also set to zero (the coarse correction starts from 0).
// PF / PC: the fine / coarse level is a float32 level in the planar layout.
template <typename T, bool PF, bool PC>
__global__ void __launch_bounds__(NT) k_restrict(int nc, const T* __restrict__ ru, const T* __restrict__ rp,
                                                 T* __restrict__ fc, T* __restrict__ gc, T* __restrict__ uc,
                                                 T* __restrict__ pc, int dom) {
    pdl_wait();
    const int n = nc;
    CELL_INDEX
    if (!active) return;
    const XferLayout lay = xfer_layout(nc, PF, PC);
    restrict_cell<true, T, PF, PC>(i, j, nc, ru, rp, fc, gc, lay, dom);
    if (uc) {
        const CellNodes cn = cell_nodes(i, j, nc);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const int k = lat_at<PC>(X, Y, lay.ldc, lay.psc);
            uc[k] = T(0);
            uc[lay.n2c + k] = T(0);
        }
        pc[j * lay.ldpc + i] = T(0);
    }
    pdl_trigger();
}

template <typename T>
void launch_restrict(cudaStream_t s, int nc, const T* ru, const T* rp, T* fc, T* gc, T* uc, T* pc, int dom) {
    launch_pdl(k_restrict<T, false, false>, cells_grid(nc), dim3(BX, BY), 0, s, nc, ru, rp, fc, gc, uc, pc, dom);
}

void launch_restrict_planar(cudaStream_t s, int nc, bool pc_planar, const float* ru, const float* rp, float* fc,
                            float* gc, float* uc, float* pc) {
    if (pc_planar)
        launch_pdl(k_restrict<float, true, true>, cells_grid(nc), dim3(BX, BY), 0, s, nc, ru, rp, fc, gc, uc, pc,
                   (int)kDomSquare);
    else
        launch_pdl(k_restrict<float, true, false>, cells_grid(nc), dim3(BX, BY), 0, s, nc, ru, rp, fc, gc, uc, pc,
                   (int)kDomSquare);
}

// Prolongation (Sec. 3, canonical embedding): every fine point owned by coarse square (I, J) is
// the coarse P2 function of that square evaluated there; P1 values are vertex injection and
// averages along coarse edges.
template <bool LDG, typename T, bool PF = false, bool PC = false>
__device__ __forceinline__ void prolong_cell(int i, int j, int nc, const T* __restrict__ uc, const T* __restrict__ pc,
                                             T* __restrict__ u, T* __restrict__ p, const XferLayout& lay,
                                             int dom = kDomSquare) {
    const int nf = 2 * nc;
    if (i < nc && j < nc) {
        T z[2][9];
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int k = lat_at<PC>(2 * i + m % 3, 2 * j + m / 3, lay.ldc, lay.psc);
            z[0][m] = ldv<LDG>(uc + k);
            z[1][m] = ldv<LDG>(uc + lay.n2c + k);
        }
        const int o = orient(i, j, nc);
#pragma unroll
        for (int fb = 0; fb < 4; ++fb)
#pragma unroll
            for (int fa = 0; fa < 4; ++fa) {
                const int X = 4 * i + fa, Y = 4 * j + fb;
                if (!interior2(X, Y, nf) || (dom == kDomL && l_masked_node(X, Y, nf))) continue;
                T sx = T(0), sy = T(0);
#pragma unroll
                for (int L = 0; L < 9; ++L) {
                    const T w = W2<T>(o, L, fb, fa);
                    sx = fma(w, z[0][L], sx);
                    sy = fma(w, z[1][L], sy);
                }
                const int k = lat_at<PF>(X, Y, lay.ldf, lay.psf);
                u[k] += sx;
                u[lay.n2f + k] += sy;
            }
    }
    const int ldp = lay.ldpc, ldpf = lay.ldpf;
    auto P = [&](int a, int b) { return ldv<LDG>(pc + (b * ldp + a)); };
    const T p00 = P(i, j);
    // on the L, fine vertices strictly inside the removed quadrant keep their zero
    auto live = [&](int x, int y) { return !(dom == kDomL && l_masked_vertex(x, y, nf)); };
    if (live(2 * i, 2 * j)) p[(2 * j) * ldpf + 2 * i] += p00;
    if (i < nc && live(2 * i + 1, 2 * j)) p[(2 * j) * ldpf + 2 * i + 1] += T(0.5) * (p00 + P(i + 1, j));
    if (j < nc && live(2 * i, 2 * j + 1)) p[(2 * j + 1) * ldpf + 2 * i] += T(0.5) * (p00 + P(i, j + 1));
    if (i < nc && j < nc && live(2 * i + 1, 2 * j + 1)) {
        const T d = orient(i, j, nc) == 0 ? p00 + P(i + 1, j + 1) : P(i + 1, j) + P(i, j + 1);
        p[(2 * j + 1) * ldpf + 2 * i + 1] += T(0.5) * d;
    }
}

template <typename T, bool PF, bool PC>
__global__ void __launch_bounds__(NT) k_prolong(int nc, const T* __restrict__ uc, const T* __restrict__ pc,
                                                T* __restrict__ u, T* __restrict__ p, int dom) {
    pdl_wait();
    const int n = nc;
    CELL_INDEX
    if (!active) return;
    prolong_cell<true, T, PF, PC>(i, j, nc, uc, pc, u, p, xfer_layout(nc, PF, PC), dom);
    pdl_trigger();
}

template <typename T>
void launch_prolong_add(cudaStream_t s, int nc, const T* uc, const T* pc, T* u, T* p, int dom) {
    launch_pdl(k_prolong<T, false, false>, cells_grid(nc), dim3(BX, BY), 0, s, nc, uc, pc, u, p, dom);
}

void launch_prolong_add_planar(cudaStream_t s, int nc, bool pc_planar, const float* uc, const float* pc, float* u,
                               float* p) {
    if (pc_planar)
        launch_pdl(k_prolong<float, true, true>, cells_grid(nc), dim3(BX, BY), 0, s, nc, uc, pc, u, p, (int)kDomSquare);
    else
        launch_pdl(k_prolong<float, true, false>, cells_grid(nc), dim3(BX, BY), 0, s, nc, uc, pc, u, p, (int)kDomSquare);
}

// ------------------------------------------------------------------------------------------
// Level 0 (N = 2): x = inv b with the bordered inverse; 27 unknowns (see elements.cpp).
template <typename T>
__global__ void k_coarse(const double* __restrict__ inv, const T* __restrict__ f, const T* __restrict__ g,
                         T* __restrict__ u, T* __restrict__ p) {
    pdl_wait();
    __shared__ double b[27];
    const int t = threadIdx.x;
    auto vpos = [](int t, int& c, int& k) {
        c = t / 9;
        const int r = t % 9;
        k = (1 + r / 3) * 5 + 1 + r % 3;
    };
    if (t < 27) {
        if (t < 18) {
            int c, k;
            vpos(t, c, k);
            b[t] = (double)f[c * 25 + k];
        } else {
            b[t] = (double)g[t - 18];
        }
    }
    __syncthreads();
    // zero the velocity boundary of level 0 (50 entries), then write the solution
    for (int k = t; k < 50; k += blockDim.x) {
        const int r = k % 25, X = r % 5, Y = r / 5;
        if (X == 0 || Y == 0 || X == 4 || Y == 4) u[k] = T(0);
    }
    if (t < 27) {
        double x = 0.0;
        for (int s = 0; s < 27; ++s) x = fma(inv[t * 27 + s], b[s], x);
        if (t < 18) {
            int c, k;
            vpos(t, c, k);
            u[c * 25 + k] = (T)x;
        } else {
            p[t - 18] = (T)x;
        }
    }
    pdl_trigger();
}

template <typename T>
void launch_coarse_solve(cudaStream_t s, const double* inv, const T* f, const T* g, T* u, T* p) {
    launch_pdl(k_coarse<T>, 1, 32, 0, s, inv, f, g, u, p);
}

// ------------------------------------------------------------------------------------------
// Shat = diag(B Ahat^{-1} B^T), Ahat = diag A (Sec. 6, eq. numintroduc): for vertex (i, j),
// sum over interior velocity nodes l and both components of B_{(i,j), l}^2 / A_{ll}.
__device__ double diagA_at(int X, int Y, int n, const OpCoef<double>& c) {
    double d = 0.0;
    const int sx0 = (X & 1) ? (X - 1) / 2 : X / 2 - 1, sx1 = (X & 1) ? sx0 : X / 2;
    const int sy0 = (Y & 1) ? (Y - 1) / 2 : Y / 2 - 1, sy1 = (Y & 1) ? sy0 : Y / 2;
    for (int sj = sy0; sj <= sy1; ++sj)
        for (int si = sx0; si <= sx1; ++si) {
            if (si < 0 || sj < 0 || si >= n || sj >= n) continue;
            const int a = X - 2 * si, b = Y - 2 * sj, o = orient(si, sj, n);
            d += c.A[o][3 * b + a][3 * b + a];
        }
    return d;
}

// On the L the sum runs over the L's velocity unknowns only (their B coefficients are the square's:
// all squares around such a node lie in the L), and Shat^{-1} = 0 at vertices outside the L.
template <typename T>
__global__ void __launch_bounds__(NT) k_schur(int n, const __grid_constant__ OpCoef<double> c, T* __restrict__ sinv,
                                              int dom, int vld) {
    CELL_INDEX
    if (!active) return;
    if (dom == kDomL && l_masked_vertex(i, j, n)) {
        sinv[(size_t)j * vld + i] = T(0);
        return;
    }
    double bx[5][5], by[5][5];
    for (int b = 0; b < 5; ++b)
        for (int a = 0; a < 5; ++a) bx[b][a] = by[b][a] = 0.0;
    for (int SQ = 0; SQ < 4; ++SQ) {
        const int si = i - (SQ & 1), sj = j - (SQ >> 1);
        if (si < 0 || sj < 0 || si >= n || sj >= n) continue;
        const int o = orient(si, sj, n);
        for (int m = 0; m < 9; ++m) {
            const int px = 2 * (si - i) + 2 + m % 3, py = 2 * (sj - j) + 2 + m / 3;
            bx[py][px] += c.Bx[o][SQ][m];
            by[py][px] += c.By[o][SQ][m];
        }
    }
    double s = 0.0;
    for (int py = 0; py < 5; ++py)
        for (int px = 0; px < 5; ++px) {
            const int X = 2 * i - 2 + px, Y = 2 * j - 2 + py;
            if (!interior2(X, Y, n) || (dom == kDomL && l_masked_node(X, Y, n))) continue;
            s += (bx[py][px] * bx[py][px] + by[py][px] * by[py][px]) / diagA_at(X, Y, n, c);
        }
    sinv[(size_t)j * vld + i] = (T)(1.0 / s);
}

template <typename T>
void launch_schur_diag(cudaStream_t s, int n, const OpCoef<double>& c, T* sinv, int dom, int vld) {
    k_schur<T><<<cells_grid(n), dim3(BX, BY), 0, s>>>(n, c, sinv, dom, vld > 0 ? vld : n + 1);
}

// ------------------------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(NT) k_pmean_partial(int n, const T* __restrict__ p, double* __restrict__ partial,
                                                      int dom) {
    pdl_wait();
    CELL_INDEX
    double v = 0.0;
    if (active) v = vertex_weight_dom(i, j, n, dom) * (double)p[(size_t)j * (n + 1) + i];
    const double t = block_sum2d(v, tid);
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
    pdl_trigger();
}

// p -= (w^T p) / |Omega| at the pressure unknowns; |Omega| = sum_i w_i = 1 (square) or 3/4 (L)
template <typename T>
__global__ void __launch_bounds__(NT) k_psub(int n, T* __restrict__ p, const double* __restrict__ scalar, int dom) {
    pdl_wait();
    CELL_INDEX
    if (!active) return;
    if (dom == kDomL) {
        if (!l_masked_vertex(i, j, n)) p[(size_t)j * (n + 1) + i] -= (T)(*scalar / 0.75);
    } else {
        p[(size_t)j * (n + 1) + i] -= (T)(*scalar);
    }
    pdl_trigger();
}

__global__ void k_reduce(const double* __restrict__ partial, int count, double* __restrict__ out) {
    pdl_wait();
    // fixed-order tree: deterministic for a given count
    __shared__ double red[1024];
    double s = 0.0;
    for (int k = threadIdx.x; k < count; k += blockDim.x) s += partial[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
    pdl_trigger();
}

cudaError_t launch_reduce(cudaStream_t s, const double* partial, int count, double* out) {
    return launch_pdl(k_reduce, 1, 1024, 0, s, partial, count, out);
}

template <typename T>
void launch_pmean(cudaStream_t s, int n, T* p, double* partial, double* scalar, int dom) {
    const dim3 grid = cells_grid(n), blk(BX, BY);
    launch_pdl(k_pmean_partial<T>, grid, blk, 0, s, n, p, partial, dom);
    launch_pdl(k_reduce, 1, 1024, 0, s, partial, grid.x * grid.y, scalar);
    launch_pdl(k_psub<T>, grid, blk, 0, s, n, p, scalar, dom);
}

template <typename T>
void launch_psub(cudaStream_t s, int n, T* p, const double* scalar, int dom) {
    launch_pdl(k_psub<T>, cells_grid(n), dim3(BX, BY), 0, s, n, p, scalar, dom);
}
template void launch_psub<double>(cudaStream_t, int, double*, const double*, int);

// ------------------------------------------------------------------------------------------
// load vectors (data f, g of Sec. 1 given by nodal values)
template <typename T>
__device__ __forceinline__ void mp_row(int i, int j, int n, const MassCoef<T>& m, const T* __restrict__ gn,
                                       T& mg, double& w) {
    mg = T(0);
    w = 0.0;
#pragma unroll
    for (int SQ = 0; SQ < 4; ++SQ) {
        const int si = i - (SQ & 1), sj = j - (SQ >> 1);
        if (si < 0 || sj < 0 || si >= n || sj >= n) continue;
        const int o = orient(si, sj, n);
        T q[4];
        load_sq_p(gview(gn, n + 1), si, sj, q);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            mg = fma(m.MP[o][SQ][r], q[r], mg);
            w += (double)m.MP[o][SQ][r];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_load(int n, const __grid_constant__ MassCoef<T> m, const __grid_constant__ OpCoef<T> c,
                                             const T* __restrict__ fn, const T* __restrict__ gn,
                                             T* __restrict__ f, T* __restrict__ g, double* __restrict__ partial) {
    CELL_INDEX
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    double wg = 0.0;
    if (active) {
        Acc<T> a;
        cell_apply<true, false, false, false, false>(i, j, n, m.M, c, gview(fn, 2 * n + 1), gview(fn + n2, 2 * n + 1), gview((const T*)nullptr, n + 1), a);
        const CellNodes cn = cell_nodes(i, j, n);
        const int ld = 2 * n + 1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const size_t k = (size_t)Y * ld + X;
            const bool unk = slot_unknown(cn, s);
            f[k] = unk ? a.au[0][s] : T(0);
            f[n2 + k] = unk ? a.au[1][s] : T(0);
        }
        T mg;
        double w;
        mp_row(i, j, n, m, gn, mg, w);
        const size_t vi = (size_t)j * (n + 1) + i;
        g[vi] = mg;
        wg = w * (double)gn[vi];
    }
    const double t = block_sum2d(wg, tid);
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_gproj(int n, const __grid_constant__ MassCoef<T> m, T* __restrict__ g,
                                              const double* __restrict__ scalar) {
    CELL_INDEX
    if (!active) return;
    double w = 0.0;
#pragma unroll
    for (int SQ = 0; SQ < 4; ++SQ) {
        const int si = i - (SQ & 1), sj = j - (SQ >> 1);
        if (si < 0 || sj < 0 || si >= n || sj >= n) continue;
        const int o = orient(si, sj, n);
#pragma unroll
        for (int r = 0; r < 4; ++r) w += (double)m.MP[o][SQ][r];
    }
    // M_P (g - c 1) = M_P g - c w,  c = int g_h = sum_i w_i g_i
    g[(size_t)j * (n + 1) + i] -= (T)(w * (*scalar));
}

template <typename T>
void launch_load(cudaStream_t s, int n, const MassCoef<T>& m, const T* fn, const T* gn, T* f, T* g,
                 int project_g, double* partial, double* scalar) {
    const dim3 grid = cells_grid(n), blk(BX, BY);
    OpCoef<T> dummy{};
    k_load<T><<<grid, blk, 0, s>>>(n, m, dummy, fn, gn, f, g, partial);
    if (project_g) {
        launch_pdl(k_reduce, 1, 1024, 0, s, partial, grid.x * grid.y, scalar);
        k_gproj<T><<<grid, blk, 0, s>>>(n, m, g, scalar);
    }
}

__global__ void __launch_bounds__(NT) k_mass_dot(int n, const __grid_constant__ MassCoef<double> m,
                                                 const __grid_constant__ OpCoef<double> c,
                                                 const double* __restrict__ av, const double* __restrict__ bv,
                                                 double* __restrict__ partial) {
    CELL_INDEX
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    double acc = 0.0;
    if (active) {
        Acc<double> a;
        cell_apply<true, false, false, false, true>(i, j, n, m.M, c, gview(bv, 2 * n + 1), gview(bv + n2, 2 * n + 1), gview((const double*)nullptr, n + 1), a);
        const CellNodes cn = cell_nodes(i, j, n);
        const int ld = 2 * n + 1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_unknown(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const size_t k = (size_t)Y * ld + X;
            acc += av[k] * a.au[0][s] + av[n2 + k] * a.au[1][s];
        }
    }
    const double t = block_sum2d(acc, tid);
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

void launch_mass_dot(cudaStream_t s, int n, const MassCoef<double>& m, const double* a, const double* b,
                     double* partial) {
    OpCoef<double> dummy{};
    k_mass_dot<<<cells_grid(n), dim3(BX, BY), 0, s>>>(n, m, dummy, a, b, partial);
}

__global__ void __launch_bounds__(NT) k_rhs_norm(int n, const double* __restrict__ f, const double* __restrict__ g,
                                                 double* __restrict__ partial) {
    CELL_INDEX
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    double ss = 0.0;
    if (active) {
        const CellNodes cn = cell_nodes(i, j, n);
        const int ld = 2 * n + 1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_unknown(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const size_t k = (size_t)Y * ld + X;
            ss += f[k] * f[k] + f[n2 + k] * f[n2 + k];
        }
        const double v = g[(size_t)j * (n + 1) + i];
        ss += v * v;
    }
    const double t = block_sum2d(ss, tid);
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

void launch_rhs_norm(cudaStream_t s, int n, const double* f, const double* g, double* partial) {
    k_rhs_norm<<<cells_grid(n), dim3(BX, BY), 0, s>>>(n, f, g, partial);
}

__global__ void __launch_bounds__(NT) k_sum_partial(int n, const double* __restrict__ g, double* __restrict__ partial) {
    CELL_INDEX
    const double v = active ? g[(size_t)j * (n + 1) + i] : 0.0;
    const double t = block_sum2d(v, tid);
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_sub_w(int n, double* __restrict__ g, const double* __restrict__ scalar) {
    CELL_INDEX
    if (!active) return;
    g[(size_t)j * (n + 1) + i] -= (*scalar) * vertex_weight(i, j, n);   // sum_i w_i = 1
}

void launch_make_consistent(cudaStream_t s, int n, double* g, double* partial, double* scalar) {
    const dim3 grid = cells_grid(n), blk(BX, BY);
    k_sum_partial<<<grid, blk, 0, s>>>(n, g, partial);
    launch_pdl(k_reduce, 1, 1024, 0, s, partial, grid.x * grid.y, scalar);
    k_sub_w<<<grid, blk, 0, s>>>(n, g, scalar);
}

__global__ void k_add_f32(size_t count, const float* __restrict__ e, double* __restrict__ x) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x)
        x[k] += (double)e[k];
}

void launch_add_f32(cudaStream_t s, size_t count, const float* e, double* x) {
    const int blocks = (int)((count + 255) / 256 < 152 * 16 ? (count + 255) / 256 : 152 * 16);
    k_add_f32<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(count, e, x);
}

// compact (2N+1)^2 x 2 / (N+1)^2 float32 state <-> the planar layout (common.cuh)
__global__ void k_to_planar(int n, const float* __restrict__ u, const float* __restrict__ p, float* __restrict__ pu,
                            float* __restrict__ pp) {
    const int ld = 2 * n + 1, n2 = ld * ld, P = pl_pitch(n), RP = pl_rows(n), vp = pl_vpitch(n);
    const int slots = 2 * RP * P, verts = (n + 1) * vp;
    const int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < slots; k += stride) {
        const int q = k % P, Y = (k / P) % RP, X = 2 * q + k / (P * RP);
        float2 v = make_float2(0.f, 0.f);
        if (interior2(X, Y, n)) v = make_float2(u[Y * ld + X], u[n2 + Y * ld + X]);
        reinterpret_cast<float2*>(pu)[k] = v;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < verts; k += stride) {
        const int i = k % vp, j = k / vp;
        pp[k] = i <= n ? p[j * (n + 1) + i] : 0.f;
    }
}

__global__ void k_from_planar(int n, const float* __restrict__ pu, const float* __restrict__ pp, float* __restrict__ u,
                              float* __restrict__ p) {
    const int ld = 2 * n + 1, n2 = ld * ld, vp = pl_vpitch(n);
    const int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += stride) {
        const int X = k % ld, Y = k / ld, o = pl_u(n, X, Y);
        u[k] = pu[o];
        u[n2 + k] = pu[o + 1];
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (n + 1) * (n + 1); k += stride) {
        const int i = k % (n + 1), j = k / (n + 1);
        p[k] = pp[j * vp + i];
    }
}

void launch_to_planar(cudaStream_t s, int n, const float* u, const float* p, float* pu, float* pp) {
    const int work = 2 * pl_rows(n) * pl_pitch(n);
    k_to_planar<<<std::min((work + 255) / 256, 4096), 256, 0, s>>>(n, u, p, pu, pp);
}

void launch_from_planar(cudaStream_t s, int n, const float* pu, const float* pp, float* u, float* p) {
    const int work = (2 * n + 1) * (2 * n + 1);
    k_from_planar<<<std::min((work + 255) / 256, 4096), 256, 0, s>>>(n, pu, pp, u, p);
}

// On the L: zero the entries of velocity arrays at nodes outside the L's unknowns' closure (the closed
// removed quadrant) and of vertex arrays at vertices strictly inside it; either pointer pair may be null.
__global__ void k_mask_l(int n, double* __restrict__ u, double* __restrict__ p) {
    const int ld = 2 * n + 1, n2 = ld * ld;
    const int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += stride) {
        const int X = k % ld, Y = k / ld;
        if (l_masked_node(X, Y, n) && u) {
            u[k] = 0.0;
            u[n2 + k] = 0.0;
        }
        if (p && X <= n && Y <= n && l_masked_vertex(X, Y, n)) p[Y * (n + 1) + X] = 0.0;
    }
}

void launch_mask_l(cudaStream_t s, int n, double* u, double* p) {
    const int ld = 2 * n + 1;
    const int blocks = std::min((ld * ld + 255) / 256, 4096);
    k_mask_l<<<blocks, 256, 0, s>>>(n, u, p);
}

#include "coarse_cycle.cuh"

// ------------------------------------------------------------------------------------------
#define INST(T)                                                                                         \
    template void launch_uzawa<T>(cudaStream_t, int, const OpCoef<T>&, T, T, T*, T*, const T*, const T*, \
                                  const T*, T*, T*, int, int, int);                                                 \
    template void launch_normal_eq<T>(cudaStream_t, int, const OpCoef<T>&, T, T*, T*, const T*, const T*, \
                                      const T*, T*, T*);                                                  \
    template void launch_restrict<T>(cudaStream_t, int, const T*, const T*, T*, T*, T*, T*, int);                 \
    template void launch_prolong_add<T>(cudaStream_t, int, const T*, const T*, T*, T*, int);              \
    template void launch_coarse_solve<T>(cudaStream_t, const double*, const T*, const T*, T*, T*);        \
    template void launch_schur_diag<T>(cudaStream_t, int, const OpCoef<double>&, T*, int, int);           \
    template void launch_pmean<T>(cudaStream_t, int, T*, double*, double*, int);                          \
    template void launch_load<T>(cudaStream_t, int, const MassCoef<T>&, const T*, const T*, T*, T*, int,  \
                                 double*, double*);
INST(float)
INST(double)
template void launch_residual<double, double>(cudaStream_t, int, const OpCoef<double>&, const double*,
                                              const double*, const double*, const double*, double*, double*,
                                              double*, float*, float*, int);
template void launch_residual<float, float>(cudaStream_t, int, const OpCoef<float>&, const float*, const float*,
                                            const float*, const float*, float*, float*, double*, float*, float*, int);
template void launch_residual<double, float>(cudaStream_t, int, const OpCoef<double>&, const double*,
                                             const double*, const double*, const double*, float*, float*,
                                             double*, float*, float*, int);

}  // namespace smg
