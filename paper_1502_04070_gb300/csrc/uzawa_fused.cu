// uzawa_fused.cu -- one whole Uzawa smoothing step (Sec. 4) in one kernel.
//
//   u^{m-1/2} = u^{m-1} + tau Ahat^{-1} (f - A u^{m-1} - B^T p^{m-1})
//   dp        = sigma Shat^{-1} (B u^{m-1/2} - g),      p^{m} = p^{m-1} + dp
//   u^{m}     = u^{m-1/2} - tau Ahat^{-1} B^T dp
//
// A CTA owns a TX x TY tile of cells.  It stages u and p with a halo of three cells in shared
// memory, computes u^{m-1/2} on the tile plus two cells, dp on the tile plus one vertex, and the
// new (u, p) on the tile, so every HBM word of u, p, f, g, Shat^{-1} is read about once and u, p
// are written once (the halo re-reads hit L2).  The step reads (u, p) and writes (u_out, p_out):
// neighbouring tiles still need the old values as halo, so the caller ping-pongs two buffers.
#include <cstdio>

#include "cellops.cuh"
#include "kernels.cuh"

namespace smg {

// plane size padded so that the two parity planes of one row start half a bank cycle apart
// (16 words for float32, 8 doubles for float64): staging writes of consecutive X are conflict-free
template <typename T>
__host__ __device__ constexpr int pad_plane(int w) {
    return sizeof(T) == 4 ? ((w + 31) / 32) * 32 + 16 : ((w + 15) / 16) * 16 + 8;
}

template <typename T, int TX, int TY>
struct FusedTile {
    // u: cells [i0-3, i0+TX+3) -> lattice columns [2(i0-3), 2(i0+TX+3)), split by parity
    static constexpr int UWH = TX + 6, UH = 2 * (TY + 6), UPL = pad_plane<T>(UWH * UH);
    static constexpr int PW = TX + 6, PH = TY + 6;               // p: vertices [i0-3, i0+TX+3)
    // u^{m-1/2}: cells [i0-2, i0+TX+2)
    static constexpr int HWH = TX + 4, HH = 2 * (TY + 4), HPL = pad_plane<T>(HWH * HH);
    static constexpr int DW = TX + 2, DH = TY + 2;               // dp: vertices [i0-1, i0+TX+1)
    static constexpr int U_OFF = 0;                              // u_x planes, then u_y planes
    static constexpr int P_OFF = U_OFF + 4 * UPL;
    static constexpr int H_OFF = P_OFF + PW * PH;
    static constexpr int D_OFF = H_OFF + 4 * HPL;
    static constexpr int TOTAL = D_OFF + DW * DH;
    static constexpr size_t BYTES = sizeof(T) * (size_t)TOTAL;
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, (sizeof(T) == 4 ? 2 : 1)) k_uzawa_fused(int n, const __grid_constant__ OpCoef<T> c, T tau, T sigma,
                                                        const T* __restrict__ u, const T* __restrict__ p,
                                                        const T* __restrict__ f, const T* __restrict__ g,
                                                        const T* __restrict__ sinv, T* __restrict__ u_out,
                                                        T* __restrict__ p_out) {
    pdl_wait();
    using G = FusedTile<T, TX, TY>;
    constexpr int NTH = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sU = sm + G::U_OFF;
    T* sP = sm + G::P_OFF;
    T* sH = sm + G::H_OFF;
    T* sD = sm + G::D_OFF;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int ld = 2 * n + 1;
    const int n2 = ld * ld;   // < 2^31 for every supported level

    // ---- stage u (both components) and p with their halos; zero outside / on the boundary.
    // Global reads run along X (coalesced); the parity split sends even / odd X to the two planes.
    const int X0 = 2 * (i0 - 3), Y0 = 2 * (j0 - 3);
    constexpr int UW = 2 * G::UWH;
    for (int q = tid; q < UW * G::UH; q += NTH) {
        const int x = q % UW, y = q / UW;
        const int X = X0 + x, Y = Y0 + y;
        T vx = T(0), vy = T(0);
        if (interior2(X, Y, n)) {
            const int k = Y * ld + X;
            vx = __ldg(u + k);
            vy = __ldg(u + n2 + k);
        }
        const int o = (x & 1) * G::UPL + y * G::UWH + (x >> 1);
        sU[o] = vx;
        sU[2 * G::UPL + o] = vy;
    }
    for (int q = tid; q < G::PW * G::PH; q += NTH) {
        const int x = q % G::PW, y = q / G::PW;
        const int I = i0 - 3 + x, J = j0 - 3 + y;
        sP[q] = (I >= 0 && J >= 0 && I <= n && J <= n) ? __ldg(p + (J * (n + 1) + I)) : T(0);
    }
    __syncthreads();

    using ULat = SLat<T, G::UWH, G::UPL>;
    using HLat = SLat<T, G::HWH, G::HPL>;
    const ULat vux{sU, i0 - 3, Y0}, vuy{sU + 2 * G::UPL, i0 - 3, Y0};
    const SVert<T, G::PW> vp{sP, i0 - 3, j0 - 3};

    // ---- u^{m-1/2} on cells [i0-2, i0+TX+2) x [j0-2, j0+TY+2)
    const int HY0 = 2 * (j0 - 2);
    for (int q = tid; q < (TX + 4) * (TY + 4); q += NTH) {
        const int ci = i0 - 2 + q % (TX + 4), cj = j0 - 2 + q / (TX + 4);
        T hx[4] = {T(0), T(0), T(0), T(0)}, hy[4] = {T(0), T(0), T(0), T(0)};
        if (ci >= 0 && cj >= 0 && ci <= n && cj <= n) {
            Acc<T> a;
            cell_apply_auto<true, true, false, true, false>(ci, cj, n, c, vux, vuy, vp, a);
            const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!slot_unknown(cn, s)) continue;
                int X, Y;
                slot_pos(ci, cj, s, X, Y);
                const int k = Y * ld + X;
                const T w = tau * a.idg[s];
                hx[s] = vux.at(ci, cj, s & 1, s >> 1) + w * (__ldg(f + k) - a.au[0][s] - a.bt[0][s]);
                hy[s] = vuy.at(ci, cj, s & 1, s >> 1) + w * (__ldg(f + n2 + k) - a.au[1][s] - a.bt[1][s]);
            }
        }
        const int hc = ci - (i0 - 2), hy0 = 2 * cj - HY0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int o = (s & 1) * G::HPL + (hy0 + (s >> 1)) * G::HWH + hc;
            sH[o] = hx[s];
            sH[2 * G::HPL + o] = hy[s];
        }
    }
    __syncthreads();

    const HLat vhx{sH, i0 - 2, HY0}, vhy{sH + 2 * G::HPL, i0 - 2, HY0};

    // ---- dp on vertices [i0-1, i0+TX+1) x [j0-1, j0+TY+1)
    for (int q = tid; q < G::DW * G::DH; q += NTH) {
        const int vi = i0 - 1 + q % G::DW, vj = j0 - 1 + q / G::DW;
        T d = T(0);
        if (vi >= 0 && vj >= 0 && vi <= n && vj <= n) {
            Acc<T> a;
            cell_apply_auto<false, false, true, false, false>(vi, vj, n, c, vhx, vhy, vp, a);
            const int k = vj * (n + 1) + vi;
            d = sigma * __ldg(sinv + k) * (a.bu - __ldg(g + k));
        }
        sD[q] = d;
    }
    __syncthreads();

    // ---- new (u, p) on the owned tile
    const int ci = i0 + threadIdx.x, cj = j0 + threadIdx.y;
    if (ci > n || cj > n) return;
    const SVert<T, G::DW> vd{sD, i0 - 1, j0 - 1};
    Acc<T> a;
    cell_apply_auto<false, true, false, true, false>(ci, cj, n, c, vhx, vhy, vd, a);
    const CellNodes cn = cell_nodes(ci, cj, n);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (!slot_exists(cn, s)) continue;
        int X, Y;
        slot_pos(ci, cj, s, X, Y);
        const int k = Y * ld + X;
        T ox = T(0), oy = T(0);
        if (slot_unknown(cn, s)) {
            const T w = tau * a.idg[s];
            ox = vhx.at(ci, cj, s & 1, s >> 1) - w * a.bt[0][s];
            oy = vhy.at(ci, cj, s & 1, s >> 1) - w * a.bt[1][s];
        }
        u_out[k] = ox;
        u_out[n2 + k] = oy;
    }
    p_out[cj * (n + 1) + ci] = vp(ci, cj) + vd(ci, cj);
    pdl_trigger();
}

// Step variants the autotuner chooses from, per level, for float32 (float64 uses the three-kernel
// step).  Fused one-kernel tiles (TX x TY cells): 0: 32 x 16, 1: 32 x 8, 2: 64 x 8, 3: 16 x 16.
// Three-kernel step (one thread per cell and phase, no halo recomputation; short per-thread work
// suits the small levels, whose few fused tiles are issue-bound) with blocks 4: 32 x 8, 5: 16 x 8,
// 6: 8 x 8.  Fused step on component-pair tiles with packed FP32x2 arithmetic (uzawa_pair.cu):
// 7: 28 cells wide, 8 warps, height chosen per level; 8: the same with 4 warps; 9: 28 x 8 cells,
// 12 warps (one row of the u^{m-1/2} region per warp: shortest CTAs, for small levels).  Fused step
// with the coefficients in registers and asynchronous staging (uzawa_reg.cu), 28 cells wide, 8 warps,
// height chosen per level: 10: at least 2 CTAs per SM, 11: at least 4 (shorter tiles, 64 registers).
constexpr int kFusedVariants = 4;
constexpr int kPairVariant0 = 7;
constexpr int kRegVariant0 = 10;
constexpr int kStepVariants = 12;
// per level k (N = 2^(k+1)): chosen variant; until tuned, the three-kernel step below N = 128 and the
// 32 x 16 fused tile from N = 128 up
static int g_tile_choice[32] = {5, 5, 5, 5, 5, 5, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,
                                0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
static bool g_tuned[32] = {};

static int level_of(int n) {
    int k = 0;
    while ((2 << k) < n) ++k;
    return k < 32 ? k : 31;
}

template <typename T, int TX, int TY>
static cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_uzawa_fused<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FusedTile<T, TX, TY>::BYTES);
}

template <typename T>
cudaError_t prepare_uzawa_fused() {
    if constexpr (sizeof(T) == 4) {
        cudaError_t e;
        if ((e = set_smem_attr<T, 32, 16>()) != cudaSuccess) return e;
        if ((e = set_smem_attr<T, 32, 8>()) != cudaSuccess) return e;
        if ((e = set_smem_attr<T, 64, 8>()) != cudaSuccess) return e;
        return set_smem_attr<T, 16, 16>();
    } else {
        return set_smem_attr<T, 32, 8>();
    }
}
template cudaError_t prepare_uzawa_fused<float>();
template cudaError_t prepare_uzawa_fused<double>();

template <typename T, int TX, int TY>
static void launch_v(cudaStream_t s, int n, const OpCoef<T>& c, T tau, T sigma, const T* u, const T* p, const T* f,
                     const T* g, const T* sinv, T* u_out, T* p_out) {
    using G = FusedTile<T, TX, TY>;
    const dim3 grid((n + 1 + TX - 1) / TX, (n + 1 + TY - 1) / TY), blk(TX, TY);
    launch_pdl(k_uzawa_fused<T, TX, TY>, grid, blk, G::BYTES, s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
}

template <typename T>
static void launch_variant(int v, cudaStream_t s, int n, const OpCoef<T>& c, T tau, T sigma, const T* u, const T* p,
                           const T* f, const T* g, const T* sinv, T* u_out, T* p_out) {
    if constexpr (sizeof(T) == 4) {
        switch (v) {
            case 1: launch_v<T, 32, 8>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out); return;
            case 2: launch_v<T, 64, 8>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out); return;
            case 3: launch_v<T, 16, 16>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out); return;
            default: launch_v<T, 32, 16>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out); return;
        }
    } else {
        launch_v<T, 32, 8>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
    }
}

static bool launch_step_variant(int v, cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma,
                                float* u, float* p, const float* f, const float* g, const float* sinv, float* u_out,
                                float* p_out) {
    if (v < kFusedVariants) {
        launch_variant<float>(v, s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
        return true;
    }
    if (v >= kRegVariant0) {
        // the register tile checks the level's coefficients against its compile-time structure; if
        // they do not match, the pair tile runs instead
        if (!launch_uzawa_reg(v - kRegVariant0, s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out))
            launch_uzawa_pair(0, s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
        return true;
    }
    if (v >= kPairVariant0) {
        launch_uzawa_pair(v - kPairVariant0, s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
        return true;
    }
    const int bx = v == 4 ? 32 : (v == 5 ? 16 : 8), by = 8;
    launch_uzawa<float>(s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out, bx, by);
    return false;
}

template <typename T>
cudaError_t launch_uzawa_fused(cudaStream_t s, int n, const OpCoef<T>& c, T tau, T sigma, const T* u, const T* p,
                               const T* f, const T* g, const T* sinv, T* u_out, T* p_out) {
    launch_variant<T>(sizeof(T) == 4 ? g_tile_choice[level_of(n)] : 0, s, n, c, tau, sigma, u, p, f, g, sinv,
                      u_out, p_out);
    return cudaSuccess;
}

// Times every tile shape on the given level buffers (the step is applied to (u, p) -> (u_out, p_out)
// repeatedly; the caller's data are overwritten) and keeps the fastest for this level size.
cudaError_t autotune_uzawa_fused(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, float* u,
                                 float* p, const float* f, const float* g, const float* sinv, float* u_out,
                                 float* p_out, int* chosen, float* best_ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cudaErrorUnknown;
    int best = 0;
    float bms = 1e30f;
    const int reps = n >= 512 ? 5 : 20;
    for (int v = 0; v < kStepVariants; ++v) {
        bool sw = launch_step_variant(v, s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r) {
            float *xu = sw ? u_out : u, *xp = sw ? p_out : p, *ou = sw ? u : u_out, *op = sw ? p : p_out;
            if (launch_step_variant(v, s, n, c, tau, sigma, xu, xp, f, g, sinv, ou, op)) sw = !sw;
        }
        cudaEventRecord(e1, s);
        cudaError_t err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return err;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < bms) {
            bms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_tile_choice[level_of(n)] = best;
    g_tuned[level_of(n)] = true;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = bms;
    return cudaGetLastError();
}

bool uzawa_tuned(int n) { return g_tuned[level_of(n)]; }
int uzawa_choice(int n) { return g_tile_choice[level_of(n)]; }
bool set_uzawa_choice(int n, int v) {
    if (v < 0 || v >= kStepVariants) return false;
    g_tile_choice[level_of(n)] = v;
    g_tuned[level_of(n)] = true;
    return true;
}

bool launch_uzawa_auto(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, float* u, float* p,
                       const float* f, const float* g, const float* sinv, float* u_out, float* p_out) {
    return launch_step_variant(g_tile_choice[level_of(n)], s, n, c, tau, sigma, u, p, f, g, sinv, u_out, p_out);
}

template cudaError_t launch_uzawa_fused<float>(cudaStream_t, int, const OpCoef<float>&, float, float, const float*,
                                               const float*, const float*, const float*, const float*, float*, float*);
template cudaError_t launch_uzawa_fused<double>(cudaStream_t, int, const OpCoef<double>&, double, double,
                                                const double*, const double*, const double*, const double*,
                                                const double*, double*, double*);

}  // namespace smg
