// coarse_cycle.cuh -- the float32 V-cycle below a small level in ONE launch (included by kernels.cu).
//
// On levels with N <= 32 a multigrid step is a few thousand cells: one launch per phase would
// spend far more time in launch latency and in a handful of busy SMs than in arithmetic.  Here one
// CTA keeps every array of levels 0..LC (LC <= 4) in shared memory (about 161 KB for LC = 4) and
// runs the whole cycle of Sec. 3 on them -- nu_pre Uzawa steps, residual, restriction, the exact
// level-0 solve, prolongation, nu_post Uzawa steps on every level -- with CTA barriers between the
// phases.  The arithmetic is the same as the per-level kernels (same cell functions).

constexpr int kCoarseTop = kCoarseCycleTop;   // deepest level handled in shared memory (N = 32)
constexpr int kCoarseThreads = 512;

// value at lattice point / vertex of a dense shared-memory array with row length ld
template <typename T>
struct PView {
    static constexpr bool zero_filled = false;
    const T* p;
    int ld;
    __device__ __forceinline__ T operator()(int X, int Y) const { return p[Y * ld + X]; }
    __device__ __forceinline__ T at(int si, int sj, int a, int b) const { return p[(2 * sj + b) * ld + 2 * si + a]; }
};

__host__ __device__ constexpr int cc_n2(int l) { return ((4 << l) + 1) * ((4 << l) + 1); }
__host__ __device__ constexpr int cc_n1(int l) { return ((2 << l) + 1) * ((2 << l) + 1); }
// floats of one level: u, f, tu (2 n2 each), p, g, tp, sinv (n1 each)
__host__ __device__ constexpr int cc_level_floats(int l) { return 6 * cc_n2(l) + 4 * cc_n1(l); }
__host__ __device__ constexpr int cc_floats(int top) {
    return top < 0 ? 0 : cc_level_floats(top) + cc_floats(top - 1);
}
inline size_t coarse_cycle_smem(int top) { return sizeof(float) * (size_t)cc_floats(top) + 64 * sizeof(double); }

struct CCLevel {
    float *u, *f, *tu, *p, *g, *tp, *sv;
    int n;
};

__device__ __forceinline__ CCLevel cc_level(float* base, int l) {
    int off = 0;
    for (int k = 0; k < l; ++k) off += cc_level_floats(k);
    CCLevel L;
    const int n2 = cc_n2(l), n1 = cc_n1(l);
    L.n = 2 << l;
    L.u = base + off;
    L.f = L.u + 2 * n2;
    L.tu = L.f + 2 * n2;
    L.p = L.tu + 2 * n2;
    L.g = L.p + n1;
    L.tp = L.g + n1;
    L.sv = L.tp + n1;
    return L;
}

// one Uzawa step (Sec. 4) on a shared-memory level: u^{m-1/2} -> tu, dp -> tp, then u
__device__ void cc_smooth(const CCLevel& L, const OpCoef<float>& c, float tau, float sigma) {
    const int n = L.n, ld = 2 * n + 1, n2 = ld * ld, cells = (n + 1) * (n + 1);
    const PView<float> vux{L.u, ld}, vuy{L.u + n2, ld}, vp{L.p, n + 1};
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        const int i = q % (n + 1), j = q / (n + 1);
        Acc<float> a;
        cell_apply_auto<true, true, false, true, false>(i, j, n, c, vux, vuy, vp, a);
        const CellNodes cn = cell_nodes(i, j, n);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const int k = Y * ld + X;
            const bool unk = slot_unknown(cn, s);
            L.tu[k] = unk ? L.u[k] + tau * (L.f[k] - a.au[0][s] - a.bt[0][s]) * a.idg[s] : 0.f;
            L.tu[n2 + k] = unk ? L.u[n2 + k] + tau * (L.f[n2 + k] - a.au[1][s] - a.bt[1][s]) * a.idg[s] : 0.f;
        }
    }
    __syncthreads();
    const PView<float> vhx{L.tu, ld}, vhy{L.tu + n2, ld};
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        const int i = q % (n + 1), j = q / (n + 1);
        Acc<float> a;
        cell_apply_auto<false, false, true, false, false>(i, j, n, c, vhx, vhy, vp, a);
        const float d = sigma * L.sv[q] * (a.bu - L.g[q]);
        L.p[q] += d;
        L.tp[q] = d;
    }
    __syncthreads();
    const PView<float> vd{L.tp, n + 1};
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        const int i = q % (n + 1), j = q / (n + 1);
        Acc<float> a;
        cell_apply_auto<false, true, false, true, false>(i, j, n, c, vhx, vhy, vd, a);
        const CellNodes cn = cell_nodes(i, j, n);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const int k = Y * ld + X;
            const bool unk = slot_unknown(cn, s);
            L.u[k] = unk ? L.tu[k] - tau * a.bt[0][s] * a.idg[s] : 0.f;
            L.u[n2 + k] = unk ? L.tu[n2 + k] - tau * a.bt[1][s] * a.idg[s] : 0.f;
        }
    }
    __syncthreads();
}

// r = F - A x on a shared-memory level into (tu, tp)
__device__ void cc_residual(const CCLevel& L, const OpCoef<float>& c) {
    const int n = L.n, ld = 2 * n + 1, n2 = ld * ld, cells = (n + 1) * (n + 1);
    const PView<float> vux{L.u, ld}, vuy{L.u + n2, ld}, vp{L.p, n + 1};
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        const int i = q % (n + 1), j = q / (n + 1);
        Acc<float> a;
        cell_apply_auto<true, true, true, false, false>(i, j, n, c, vux, vuy, vp, a);
        const CellNodes cn = cell_nodes(i, j, n);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_exists(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const int k = Y * ld + X;
            const bool unk = slot_unknown(cn, s);
            L.tu[k] = unk ? L.f[k] - a.au[0][s] - a.bt[0][s] : 0.f;
            L.tu[n2 + k] = unk ? L.f[n2 + k] - a.au[1][s] - a.bt[1][s] : 0.f;
        }
        L.tp[q] = L.g[q] - a.bu;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kCoarseThreads, 1) k_coarse_cycle(const __grid_constant__ CoarseCycleArgs A) {
    pdl_enter();
    extern __shared__ __align__(16) float cc_smem[];
    double* bvec = reinterpret_cast<double*>(cc_smem);            // 27 doubles for the level-0 solve
    float* base = cc_smem + 2 * 64;                                 // after 64 doubles of scratch
    const int top = A.top;
    {   // state of the top level, its right-hand side, and Shat^{-1} of every level
        const CCLevel T = cc_level(base, top);
        const int n2 = cc_n2(top), n1 = cc_n1(top);
        for (int q = threadIdx.x; q < 2 * n2; q += blockDim.x) {
            T.u[q] = A.u[q];
            T.f[q] = A.f[q];
        }
        for (int q = threadIdx.x; q < n1; q += blockDim.x) {
            T.p[q] = A.p[q];
            T.g[q] = A.g[q];
        }
        for (int l = 1; l <= top; ++l) {
            const CCLevel L = cc_level(base, l);
            for (int q = threadIdx.x; q < cc_n1(l); q += blockDim.x) L.sv[q] = A.sinv[l - 1][q];
        }
    }
    __syncthreads();
    // down: smooth, residual, restrict (and start the coarser iterate from zero)
    for (int l = top; l >= 1; --l) {
        const CCLevel L = cc_level(base, l), C = cc_level(base, l - 1);
        const OpCoef<float>& c = A.c[l - 1];
        for (int m = 0; m < A.nu_pre; ++m) cc_smooth(L, c, A.tau, A.sigma);
        cc_residual(L, c);
        const int nc = C.n, ldc = 2 * nc + 1, n2c = ldc * ldc;
        for (int q = threadIdx.x; q < (nc + 1) * (nc + 1); q += blockDim.x) {
            const int i = q % (nc + 1), j = q / (nc + 1);
            restrict_cell<false>(i, j, nc, L.tu, L.tp, C.f, C.g);
            const CellNodes cn = cell_nodes(i, j, nc);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!slot_exists(cn, s)) continue;
                int X, Y;
                slot_pos(i, j, s, X, Y);
                C.u[Y * ldc + X] = 0.f;
                C.u[n2c + Y * ldc + X] = 0.f;
            }
            C.p[q] = 0.f;
        }
        __syncthreads();
    }
    {   // level 0: exact solve with the bordered inverse (27 unknowns, see elements.cpp)
        const CCLevel Z = cc_level(base, 0);
        const int t = threadIdx.x;
        if (t < 27) {
            if (t < 18) {
                const int cc = t / 9, r = t % 9;
                bvec[t] = (double)Z.f[cc * 25 + (1 + r / 3) * 5 + 1 + r % 3];
            } else {
                bvec[t] = (double)Z.g[t - 18];
            }
        }
        __syncthreads();
        if (t < 27) {
            double x = 0.0;
            for (int s = 0; s < 27; ++s) x = fma(A.inv[t * 27 + s], bvec[s], x);
            if (t < 18) {
                const int cc = t / 9, r = t % 9;
                Z.u[cc * 25 + (1 + r / 3) * 5 + 1 + r % 3] = (float)x;
            } else {
                Z.p[t - 18] = (float)x;
            }
        }
        __syncthreads();
    }
    // up: prolongate and correct, smooth
    for (int l = 1; l <= top; ++l) {
        const CCLevel L = cc_level(base, l), C = cc_level(base, l - 1);
        const int nc = C.n;
        for (int q = threadIdx.x; q < (nc + 1) * (nc + 1); q += blockDim.x)
            prolong_cell<false>(q % (nc + 1), q / (nc + 1), nc, C.u, C.p, L.u, L.p);
        __syncthreads();
        for (int m = 0; m < A.nu_post; ++m) cc_smooth(L, A.c[l - 1], A.tau, A.sigma);
    }
    {
        const CCLevel T = cc_level(base, top);
        for (int q = threadIdx.x; q < 2 * cc_n2(top); q += blockDim.x) A.u[q] = T.u[q];
        for (int q = threadIdx.x; q < cc_n1(top); q += blockDim.x) A.p[q] = T.p[q];
    }
}

cudaError_t prepare_coarse_cycle() {
    return cudaFuncSetAttribute(k_coarse_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarse_cycle_smem(kCoarseTop));
}

void launch_coarse_cycle(cudaStream_t s, const CoarseCycleArgs& a) {
    launch_pdl(k_coarse_cycle, dim3(1), dim3(kCoarseThreads), coarse_cycle_smem(a.top), s, a);
}
