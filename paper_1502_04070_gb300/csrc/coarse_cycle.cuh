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

// The same arrays read without tests, for cells whose windows lie inside (see cc_cell).
template <typename T>
struct PViewU {
    static constexpr bool zero_filled = true;
    const T* p;
    int ld;
    __device__ __forceinline__ T operator()(int X, int Y) const { return p[Y * ld + X]; }
    __device__ __forceinline__ T at(int si, int sj, int a, int b) const { return p[(2 * sj + b) * ld + 2 * si + a]; }
};

// Work item q of a level with n cells per side -> cell (i, j) and its code path, ordered so that
// a warp mostly stays on one path: first the cells with 2 <= i, j <= n - 2 off the mid-lines,
// quadrant by quadrant (SW, NE: orientation 0, class 0; SE, NW: orientation 1, class 1), whose
// windows lie inside the lattice; then (class 2) the rows 0, 1, n/2, n - 1, n in full and the
// columns 0, 1, n/2, n - 1, n of the other rows.  Covers every cell once for n >= 4.
__device__ __forceinline__ void cc_cell(int q, int n, int& i, int& j, int& cls) {
    const int h = n >> 1, m = h - 2, nin = m * m;
    if (q < 4 * nin) {
        const int quad = q / nin, r = q - quad * nin;
        const int di = r % m, dj = r / m;
        i = (quad == 0 || quad == 3) ? 2 + di : h + 1 + di;
        j = (quad == 0 || quad == 2) ? 2 + dj : h + 1 + dj;
        cls = quad < 2 ? 0 : 1;
        return;
    }
    int r = q - 4 * nin;
    auto sel = [&](int t) { return t == 0 ? 0 : t == 1 ? 1 : t == 2 ? h : t == 3 ? n - 1 : n; };
    if (r < 5 * (n + 1)) {
        j = sel(r / (n + 1));
        i = r % (n + 1);
    } else {
        r -= 5 * (n + 1);
        const int row = r / 5;
        i = sel(r % 5);
        j = row < m ? 2 + row : h + 1 + (row - m);
    }
    cls = 2;
}

// Rows of a cell of any stencil class k, as rolled loops over the full 5 x 5 and 3 x 3 windows
// with tested reads: little code for the few cells on the boundary ring and the mid-lines (the
// whole cycle of this kernel runs on one SM, whose instruction cache it has to fit).
template <bool DA, bool DBT, bool DB, bool DD>
__device__ __noinline__ void cc_apply_rolled(int i, int j, int n, int k, const OpCoef<float>& c, const float* ux,
                                             const float* uy, const float* vp, Acc<float>& a) {
    const int ld = 2 * n + 1;
#pragma unroll
    for (int s = 0; s < 4; ++s) a.au[0][s] = a.au[1][s] = a.bt[0][s] = a.bt[1][s] = a.idg[s] = 0.f;
    a.bu = 0.f;
    if constexpr (DA || DB) {
#pragma unroll 1
        for (int w = 0; w < 25; ++w) {
            const int X = 2 * i + w % 5 - 2, Y = 2 * j + w / 5 - 2;
            if (X < 0 || Y < 0 || X > 2 * n || Y > 2 * n) continue;
            const float vx = ux[Y * ld + X], vy = uy[Y * ld + X];
            if constexpr (DA) {
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    a.au[0][s] = fmaf(c.MA[k][s][w], vx, a.au[0][s]);
                    a.au[1][s] = fmaf(c.MA[k][s][w], vy, a.au[1][s]);
                }
            }
            if constexpr (DB) a.bu = fmaf(c.MBx[k][w], vx, fmaf(c.MBy[k][w], vy, a.bu));
        }
    }
    if constexpr (DBT) {
#pragma unroll 1
        for (int v = 0; v < 9; ++v) {
            const int I = i + v % 3 - 1, J = j + v / 3 - 1;
            if (I < 0 || J < 0 || I > n || J > n) continue;
            const float pv = vp[J * (n + 1) + I];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                a.bt[0][s] = fmaf(c.MBTx[k][s][v], pv, a.bt[0][s]);
                a.bt[1][s] = fmaf(c.MBTy[k][s][v], pv, a.bt[1][s]);
            }
        }
    }
    if constexpr (DD) {
#pragma unroll
        for (int s = 0; s < 4; ++s) a.idg[s] = c.MIdg[k][s];
    }
}

// operator rows of work item q on a shared-memory level (velocity arrays ux, uy, vertex array vp)
template <bool DA, bool DBT, bool DB, bool DD>
__device__ __forceinline__ void cc_apply(int q, int n, const OpCoef<float>& c, const float* ux, const float* uy,
                                         const float* vp, int& i, int& j, Acc<float>& a) {
    int cls;
    cc_cell(q, n, i, j, cls);
    const int ld = 2 * n + 1;
    if (cls == 0) {
        cell_apply_merged<DA, DBT, DB, DD, false, 0>(i, j, n, c, PViewU<float>{ux, ld}, PViewU<float>{uy, ld},
                                                     PViewU<float>{vp, n + 1}, a);
    } else if (cls == 1) {
        cell_apply_merged<DA, DBT, DB, DD, false, 1>(i, j, n, c, PViewU<float>{ux, ld}, PViewU<float>{uy, ld},
                                                     PViewU<float>{vp, n + 1}, a);
    } else {
        cc_apply_rolled<DA, DBT, DB, DD>(i, j, n, stencil_class(i, j, n), c, ux, uy, vp, a);
    }
}

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
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        int i, j;
        Acc<float> a;
        cc_apply<true, true, false, true>(q, n, c, L.u, L.u + n2, L.p, i, j, a);
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
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        int i, j;
        Acc<float> a;
        cc_apply<false, false, true, false>(q, n, c, L.tu, L.tu + n2, L.p, i, j, a);
        const int v = j * (n + 1) + i;
        const float d = sigma * L.sv[v] * (a.bu - L.g[v]);
        L.p[v] += d;
        L.tp[v] = d;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        int i, j;
        Acc<float> a;
        cc_apply<false, true, false, true>(q, n, c, L.tu, L.tu + n2, L.tp, i, j, a);
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
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        int i, j;
        Acc<float> a;
        cc_apply<true, true, true, false>(q, n, c, L.u, L.u + n2, L.p, i, j, a);
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
        L.tp[j * (n + 1) + i] = L.g[j * (n + 1) + i] - a.bu;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kCoarseThreads, 1) k_coarse_cycle(const __grid_constant__ CoarseCycleArgs A) {
    pdl_enter();
    extern __shared__ __align__(16) float cc_smem[];
    // The operator coefficients of every level, copied from the parameter bank: the cycle indexes
    // levels at run time, and run-time-indexed parameter reads would each wait on the constant cache.
    __shared__ OpCoef<float> sc[kCoarseTop];
    double* bvec = reinterpret_cast<double*>(cc_smem);            // 27 doubles for the level-0 solve
    float* base = cc_smem + 2 * 64;                                 // after 64 doubles of scratch
    const int top = A.top;
    {
        const float* src = reinterpret_cast<const float*>(&A.c[0]);
        float* dst = reinterpret_cast<float*>(&sc[0]);
        const int words = top * (int)(sizeof(OpCoef<float>) / sizeof(float));
        for (int q = threadIdx.x; q < words; q += blockDim.x) dst[q] = src[q];
    }
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
        const OpCoef<float>& c = sc[l - 1];
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
        for (int m = 0; m < A.nu_post; ++m) cc_smooth(L, sc[l - 1], A.tau, A.sigma);
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
