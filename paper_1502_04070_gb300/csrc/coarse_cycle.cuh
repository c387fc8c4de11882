// coarse_cycle.cuh -- the float32 V-cycle below a small level in ONE launch (included by kernels.cu).
//
// On levels with N <= 32 a multigrid step is a few thousand cells: one launch per phase would
// spend far more time in launch latency and in a handful of busy SMs than in arithmetic.  Here one
// CTA keeps every array of levels 0..LC (LC <= 4) in shared memory (about 192 KB for LC = 4) and
// runs the whole cycle of Sec. 3 on them -- nu_pre Uzawa steps, residual, restriction, the exact
// level-0 solve, prolongation, nu_post Uzawa steps on every level -- with CTA barriers between the
// phases.  The arithmetic is the same as the per-level kernels (same cell functions).
//
// Every shared array carries a zero border (two lattice points around the velocity lattice, one
// vertex around the pressure grid) that nothing writes, so no window read needs a range test; the
// Dirichlet values are zeros in the arrays themselves.

constexpr int kCoarseTop = kCoarseCycleTop;   // deepest level handled in shared memory (N = 32)
constexpr int kCoarseThreads = 1024;

// value at lattice point / vertex of a padded shared-memory array (p at the (0, 0) entry)
template <typename T>
struct PViewU {
    static constexpr bool zero_filled = true;
    const T* p;
    int ld;
    __device__ __forceinline__ T operator()(int X, int Y) const { return p[Y * ld + X]; }
    __device__ __forceinline__ T at(int si, int sj, int a, int b) const { return p[(2 * sj + b) * ld + 2 * si + a]; }
};

// padded geometry of level l (N = 2^(l+1)): velocity lattice rows of 2N + 5, vertex rows of N + 3
__host__ __device__ constexpr int cc_ldu(int l) { return (4 << l) + 5; }
__host__ __device__ constexpr int cc_ldv(int l) { return (2 << l) + 3; }
__host__ __device__ constexpr int cc_n2(int l) { return cc_ldu(l) * cc_ldu(l); }
__host__ __device__ constexpr int cc_n1(int l) { return cc_ldv(l) * cc_ldv(l); }
// floats of one level: u, f, tu (2 n2 each), p, g, tp, sinv (n1 each)
__host__ __device__ constexpr int cc_level_floats(int l) { return 6 * cc_n2(l) + 4 * cc_n1(l); }
__host__ __device__ constexpr int cc_floats(int top) {
    return top < 0 ? 0 : cc_level_floats(top) + cc_floats(top - 1);
}
inline size_t coarse_cycle_smem(int top) { return sizeof(float) * (size_t)cc_floats(top) + 64 * sizeof(double); }

// one level's arrays; every pointer is at the (0, 0) entry of its padded array
struct CCLevel {
    float *u, *f, *tu, *p, *g, *tp, *sv;
    int n, ldu, n2u, ldv;
};

__device__ __forceinline__ CCLevel cc_level(float* base, int l) {
    int off = 0;
    for (int k = 0; k < l; ++k) off += cc_level_floats(k);
    CCLevel L;
    const int n2 = cc_n2(l), n1 = cc_n1(l);
    L.n = 2 << l;
    L.ldu = cc_ldu(l);
    L.n2u = n2;
    L.ldv = cc_ldv(l);
    const int ou = 2 * L.ldu + 2, ov = L.ldv + 1;
    float* q = base + off;
    L.u = q + ou;
    L.f = q + 2 * n2 + ou;
    L.tu = q + 4 * n2 + ou;
    q += 6 * n2;
    L.p = q + ov;
    L.g = q + n1 + ov;
    L.tp = q + 2 * n1 + ov;
    L.sv = q + 3 * n1 + ov;
    return L;
}

// Work item q of a level with n cells per side -> cell (i, j) and its code path, ordered so that
// a warp stays on one path: first the four quadrants off the mid-lines (SW, NE: orientation 0,
// class 0; SE, NW: orientation 1, class 1), boundary ring included (the zero border stands for
// the squares outside), then (class 2) the 2n + 1 cells on the mid-lines.
__device__ __forceinline__ void cc_cell(int q, int n, int& i, int& j, int& cls) {
    const int h = n >> 1, nq = h * h;
    if (q < 4 * nq) {
        const int quad = q / nq, r = q - quad * nq;
        const int di = r % h, dj = r / h;
        i = (quad == 0 || quad == 3) ? di : h + 1 + di;
        j = (quad == 0 || quad == 2) ? dj : h + 1 + dj;
        cls = quad < 2 ? 0 : 1;
        return;
    }
    const int m = q - 4 * nq;
    if (m <= n) {
        i = h;
        j = m;
    } else {
        const int r = m - (n + 1);
        i = r < h ? r : r + 1;
        j = h;
    }
    cls = 2;
}

// Rows of a cell of any stencil class k (known at run time) over the full 5 x 5 and 3 x 3 windows,
// zero coefficients included: one body for the five mid-line classes, so that the code stays
// within the instruction cache of the one SM that runs the whole cycle.  The loops are unrolled:
// a mid-line warp works on every phase of every level, and a rolled loop of dependent loads made
// it the slowest warp of each phase.
template <bool DA, bool DBT, bool DB, bool DD>
__device__ __noinline__ void cc_apply_dense(int i, int j, int k, const OpCoef<float>& c, const float* ux,
                                             const float* uy, int ld, const float* vp, int ldv, Acc<float>& a) {
#pragma unroll
    for (int s = 0; s < 4; ++s) a.au[0][s] = a.au[1][s] = a.bt[0][s] = a.bt[1][s] = a.idg[s] = 0.f;
    a.bu = 0.f;
    if constexpr (DA || DB) {
#pragma unroll
        for (int w = 0; w < 25; ++w) {
            const int o = (2 * j + w / 5 - 2) * ld + 2 * i + w % 5 - 2;
            const float vx = ux[o], vy = uy[o];
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
#pragma unroll
        for (int v = 0; v < 9; ++v) {
            const float pv = vp[(j + v / 3 - 1) * ldv + i + v % 3 - 1];
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
__device__ __forceinline__ void cc_apply(int q, const CCLevel& L, const OpCoef<float>& c, const float* ux,
                                         const float* uy, const float* vp, int& i, int& j, Acc<float>& a) {
    int cls;
    const int n = L.n;
    cc_cell(q, n, i, j, cls);
    if (cls == 0) {
        cell_apply_merged<DA, DBT, DB, DD, false, 0>(i, j, n, c, PViewU<float>{ux, L.ldu}, PViewU<float>{uy, L.ldu},
                                                     PViewU<float>{vp, L.ldv}, a);
    } else if (cls == 1) {
        cell_apply_merged<DA, DBT, DB, DD, false, 1>(i, j, n, c, PViewU<float>{ux, L.ldu}, PViewU<float>{uy, L.ldu},
                                                     PViewU<float>{vp, L.ldv}, a);
    } else {
        cc_apply_dense<DA, DBT, DB, DD>(i, j, stencil_class(i, j, n), c, ux, uy, L.ldu, vp, L.ldv, a);
    }
}

// one Uzawa step (Sec. 4) on a shared-memory level: u^{m-1/2} -> tu, dp -> tp, then u
__device__ void cc_smooth(const CCLevel& L, const OpCoef<float>& c, float tau, float sigma) {
    const int n = L.n, ld = L.ldu, n2 = L.n2u, cells = (n + 1) * (n + 1);
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        int i, j;
        Acc<float> a;
        cc_apply<true, true, false, true>(q, L, c, L.u, L.u + n2, L.p, i, j, a);
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
        cc_apply<false, false, true, false>(q, L, c, L.tu, L.tu + n2, L.p, i, j, a);
        const int v = j * L.ldv + i;
        const float d = sigma * L.sv[v] * (a.bu - L.g[v]);
        L.p[v] += d;
        L.tp[v] = d;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        int i, j;
        Acc<float> a;
        cc_apply<false, true, false, true>(q, L, c, L.tu, L.tu + n2, L.tp, i, j, a);
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
    const int n = L.n, ld = L.ldu, n2 = L.n2u, cells = (n + 1) * (n + 1);
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
        int i, j;
        Acc<float> a;
        cc_apply<true, true, true, false>(q, L, c, L.u, L.u + n2, L.p, i, j, a);
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
        L.tp[j * L.ldv + i] = L.g[j * L.ldv + i] - a.bu;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kCoarseThreads, 1) k_coarse_cycle(const __grid_constant__ CoarseCycleArgs A) {
    pdl_wait();
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
        // every array of every level starts at zero: borders, Dirichlet values, coarse iterates
        const int all = cc_floats(top);
        for (int q = threadIdx.x; q < all; q += blockDim.x) base[q] = 0.f;
    }
    __syncthreads();
    {   // state of the top level, its right-hand side, and Shat^{-1} of every level (dense in global)
        const CCLevel T = cc_level(base, top);
        const int ldd = 2 * T.n + 1, n2d = ldd * ldd;
        for (int q = threadIdx.x; q < 2 * n2d; q += blockDim.x) {
            const int comp = q >= n2d, r = q - comp * n2d;
            const int k = comp * T.n2u + (r / ldd) * T.ldu + r % ldd;
            T.u[k] = A.u[q];
            T.f[k] = A.f[q];
        }
        const int n1d = (T.n + 1) * (T.n + 1);
        for (int q = threadIdx.x; q < n1d; q += blockDim.x) {
            const int k = (q / (T.n + 1)) * T.ldv + q % (T.n + 1);
            T.p[k] = A.p[q];
            T.g[k] = A.g[q];
        }
        for (int l = 1; l <= top; ++l) {
            const CCLevel L = cc_level(base, l);
            for (int q = threadIdx.x; q < (L.n + 1) * (L.n + 1); q += blockDim.x)
                L.sv[(q / (L.n + 1)) * L.ldv + q % (L.n + 1)] = A.sinv[l - 1][q];
        }
    }
    __syncthreads();
    // down: smooth, residual, restrict (the coarser iterate starts from zero)
    for (int l = top; l >= 1; --l) {
        const CCLevel L = cc_level(base, l), C = cc_level(base, l - 1);
        const OpCoef<float>& c = sc[l - 1];
        for (int m = 0; m < A.nu_pre; ++m) cc_smooth(L, c, A.tau, A.sigma);
        cc_residual(L, c);
        const XferLayout lay{L.ldu, L.n2u, L.ldv, C.ldu, C.n2u, C.ldv};
        const int nc = C.n;
        for (int q = threadIdx.x; q < (nc + 1) * (nc + 1); q += blockDim.x) {
            const int i = q % (nc + 1), j = q / (nc + 1);
            restrict_cell<false>(i, j, nc, L.tu, L.tp, C.f, C.g, lay);
            const CellNodes cn = cell_nodes(i, j, nc);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!slot_exists(cn, s)) continue;
                int X, Y;
                slot_pos(i, j, s, X, Y);
                C.u[Y * C.ldu + X] = 0.f;
                C.u[C.n2u + Y * C.ldu + X] = 0.f;
            }
            C.p[j * C.ldv + i] = 0.f;
        }
        __syncthreads();
    }
    {   // level 0: exact solve with the bordered inverse (27 unknowns, see elements.cpp): the 3 x 3
        // interior lattice points of each velocity component, then the 3 x 3 vertices
        const CCLevel Z = cc_level(base, 0);
        const int t = threadIdx.x;
        if (t < 27) {
            if (t < 18) {
                const int cc = t / 9, r = t % 9;
                bvec[t] = (double)Z.f[cc * Z.n2u + (1 + r / 3) * Z.ldu + 1 + r % 3];
            } else {
                bvec[t] = (double)Z.g[((t - 18) / 3) * Z.ldv + (t - 18) % 3];
            }
        }
        __syncthreads();
        if (t < 27) {
            double x = 0.0;
            for (int s = 0; s < 27; ++s) x = fma(A.inv[t * 27 + s], bvec[s], x);
            if (t < 18) {
                const int cc = t / 9, r = t % 9;
                Z.u[cc * Z.n2u + (1 + r / 3) * Z.ldu + 1 + r % 3] = (float)x;
            } else {
                Z.p[((t - 18) / 3) * Z.ldv + (t - 18) % 3] = (float)x;
            }
        }
        __syncthreads();
    }
    // up: prolongate and correct, smooth
    for (int l = 1; l <= top; ++l) {
        const CCLevel L = cc_level(base, l), C = cc_level(base, l - 1);
        const XferLayout lay{L.ldu, L.n2u, L.ldv, C.ldu, C.n2u, C.ldv};
        const int nc = C.n;
        for (int q = threadIdx.x; q < (nc + 1) * (nc + 1); q += blockDim.x)
            prolong_cell<false>(q % (nc + 1), q / (nc + 1), nc, C.u, C.p, L.u, L.p, lay);
        __syncthreads();
        for (int m = 0; m < A.nu_post; ++m) cc_smooth(L, sc[l - 1], A.tau, A.sigma);
    }
    {
        const CCLevel T = cc_level(base, top);
        const int ldd = 2 * T.n + 1, n2d = ldd * ldd;
        for (int q = threadIdx.x; q < 2 * n2d; q += blockDim.x) {
            const int comp = q >= n2d, r = q - comp * n2d;
            A.u[q] = T.u[comp * T.n2u + (r / ldd) * T.ldu + r % ldd];
        }
        for (int q = threadIdx.x; q < (T.n + 1) * (T.n + 1); q += blockDim.x)
            A.p[q] = T.p[(q / (T.n + 1)) * T.ldv + q % (T.n + 1)];
    }
    pdl_trigger();
}

cudaError_t prepare_coarse_cycle() {
    return cudaFuncSetAttribute(k_coarse_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarse_cycle_smem(kCoarseTop));
}

void launch_coarse_cycle(cudaStream_t s, const CoarseCycleArgs& a) {
    launch_pdl(k_coarse_cycle, dim3(1), dim3(kCoarseThreads), coarse_cycle_smem(a.top), s, a);
}
