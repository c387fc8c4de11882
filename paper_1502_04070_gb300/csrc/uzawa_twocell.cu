// uzawa_twocell.cu -- the float32 three-kernel Uzawa step (Sec. 4) with two cells per thread.
//
// The same three phases as k_uzawa_u / k_uzawa_p / k_uzawa_u2 (kernels.cu), but a thread takes
// the vertically adjacent cells (i, 2t) and (i, 2t + 1).  Their 5 x 5 lattice windows share three
// rows and their 3 x 3 vertex windows share two, and when both cells have the same stencil class
// (everywhere but the row below the mid-line y = 1/2) each coefficient is read once for both.
// Blocks of 32 x 8 threads cover 32 x 16 cells.
#include "cellops.cuh"
#include "kernels.cuh"

namespace smg {

namespace {

constexpr int TBX = 32, TBY = 8;   // threads; cells per block: 32 x 16

// cells (i, j) and (i, j + 1) of one class C: the two merged rows in one basic block, so that the
// shared window values and coefficients are loaded once
template <bool DA, bool DBT, bool DB, bool DD, int C, typename VU, typename VP>
__device__ __forceinline__ void two_merged(int i, int j, int n, const OpCoef<float>& c, const VU& ux, const VU& uy,
                                           const VP& p, Acc<float>& a0, Acc<float>& a1) {
    cell_apply_merged<DA, DBT, DB, DD, false, C>(i, j, n, c, ux, uy, p, a0);
    cell_apply_merged<DA, DBT, DB, DD, false, C>(i, j + 1, n, c, ux, uy, p, a1);
}

// Rows of the thread's two cells.  Blocks at least `margin` cells inside the boundary read
// without tests (and, with margin 2, without the Dirichlet mask MASK asks for).
template <bool DA, bool DBT, bool DB, bool DD, bool MASK>
__device__ __forceinline__ void two_cells(int i, int j, int n, int margin, const OpCoef<float>& c, const float* ux,
                                          const float* uy, const float* vp, Acc<float>& a0, Acc<float>& a1) {
    const int ld = 2 * n + 1;
    const int i0 = blockIdx.x * TBX, j0 = blockIdx.y * TBY * 2;
    const bool inner = i0 >= margin && j0 >= margin && i0 + TBX - 1 <= n - margin && j0 + 2 * TBY - 1 <= n - margin;
    const int k0 = stencil_class(i, j, n), k1 = stencil_class(i, j + 1, n);
    if (inner && k0 == k1) {
        const GViewU<float> vx{ux, ld}, vy{uy, ld}, pv{vp, n + 1};
        switch (k0) {
            case 0: two_merged<DA, DBT, DB, DD, 0>(i, j, n, c, vx, vy, pv, a0, a1); break;
            case 1: two_merged<DA, DBT, DB, DD, 1>(i, j, n, c, vx, vy, pv, a0, a1); break;
            case 2: two_merged<DA, DBT, DB, DD, 2>(i, j, n, c, vx, vy, pv, a0, a1); break;
            case 3: two_merged<DA, DBT, DB, DD, 3>(i, j, n, c, vx, vy, pv, a0, a1); break;
            case 4: two_merged<DA, DBT, DB, DD, 4>(i, j, n, c, vx, vy, pv, a0, a1); break;
            case 5: two_merged<DA, DBT, DB, DD, 5>(i, j, n, c, vx, vy, pv, a0, a1); break;
            default: two_merged<DA, DBT, DB, DD, 6>(i, j, n, c, vx, vy, pv, a0, a1); break;
        }
    } else {
        const GView<float> vx{ux, ld}, vy{uy, ld}, pv{vp, n + 1};
        cell_apply_auto<DA, DBT, DB, DD, MASK>(i, j, n, c, vx, vy, pv, a0);
        if (j + 1 <= n) cell_apply_auto<DA, DBT, DB, DD, MASK>(i, j + 1, n, c, vx, vy, pv, a1);
    }
}

#define TWO_CELL_INDEX                                   \
    const int i = blockIdx.x * TBX + threadIdx.x;        \
    const int j = (blockIdx.y * TBY + threadIdx.y) * 2;  \
    if (i > n || j > n) return;

__global__ void __launch_bounds__(TBX* TBY) k_uzawa2_u(int n, const __grid_constant__ OpCoef<float> c, float tau,
                                                       const float* __restrict__ u, const float* __restrict__ p,
                                                       const float* __restrict__ f, float* __restrict__ uh) {
    pdl_enter();
    TWO_CELL_INDEX
    const int ld = 2 * n + 1, n2 = ld * ld;
    Acc<float> a[2];
    two_cells<true, true, false, true, true>(i, j, n, 2, c, u, u + n2, p, a[0], a[1]);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (j + r > n) break;
        const CellNodes cn = cell_nodes(i, j + r, n);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j + r, s, X, Y);
            const int k = Y * ld + X;
            const bool unk = slot_unknown(cn, s);
            const float w = tau * a[r].idg[s];
            uh[k] = unk ? u[k] + w * (f[k] - a[r].au[0][s] - a[r].bt[0][s]) : 0.f;
            uh[n2 + k] = unk ? u[n2 + k] + w * (f[n2 + k] - a[r].au[1][s] - a[r].bt[1][s]) : 0.f;
        }
    }
}

__global__ void __launch_bounds__(TBX* TBY) k_uzawa2_p(int n, const __grid_constant__ OpCoef<float> c, float sigma,
                                                       const float* __restrict__ uh, float* __restrict__ p,
                                                       const float* __restrict__ g, const float* __restrict__ sinv,
                                                       float* __restrict__ dp) {
    pdl_enter();
    TWO_CELL_INDEX
    const int ld = 2 * n + 1, n2 = ld * ld;
    Acc<float> a[2];
    two_cells<false, false, true, false, false>(i, j, n, 1, c, uh, uh + n2, nullptr, a[0], a[1]);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (j + r > n) break;
        const int v = (j + r) * (n + 1) + i;
        const float d = sigma * sinv[v] * (a[r].bu - g[v]);
        p[v] += d;
        dp[v] = d;
    }
}

__global__ void __launch_bounds__(TBX* TBY) k_uzawa2_u2(int n, const __grid_constant__ OpCoef<float> c, float tau,
                                                        const float* __restrict__ uh, const float* __restrict__ dp,
                                                        float* __restrict__ u) {
    pdl_enter();
    TWO_CELL_INDEX
    const int ld = 2 * n + 1, n2 = ld * ld;
    Acc<float> a[2];
    two_cells<false, true, false, true, false>(i, j, n, 1, c, nullptr, nullptr, dp, a[0], a[1]);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (j + r > n) break;
        const CellNodes cn = cell_nodes(i, j + r, n);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j + r, s, X, Y);
            const int k = Y * ld + X;
            const bool unk = slot_unknown(cn, s);
            const float w = tau * a[r].idg[s];
            u[k] = unk ? uh[k] - w * a[r].bt[0][s] : 0.f;
            u[n2 + k] = unk ? uh[n2 + k] - w * a[r].bt[1][s] : 0.f;
        }
    }
}

}  // namespace

void launch_uzawa_twocell(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, float* u, float* p,
                          const float* f, const float* g, const float* sinv, float* uh, float* dp) {
    const dim3 blk(TBX, TBY), grid((n + 1 + TBX - 1) / TBX, (n + 1 + 2 * TBY - 1) / (2 * TBY));
    launch_pdl(k_uzawa2_u, grid, blk, 0, s, n, c, tau, (const float*)u, (const float*)p, f, uh);
    launch_pdl(k_uzawa2_p, grid, blk, 0, s, n, c, sigma, (const float*)uh, p, g, sinv, dp);
    launch_pdl(k_uzawa2_u2, grid, blk, 0, s, n, c, tau, (const float*)uh, (const float*)dp, u);
}

}  // namespace smg
