// dense.cu -- the exact solve on the coarsest level of the iteration when that level is finer than
// the coarse mesh (Sec. 3: the coarse problem is solved exactly).
//
// The level-c system of eq. gen:bil:mv bordered with the zero-mean pressure condition (size nb,
// 2212 at N = 16) is inverted once per beta in float64 by Gauss-Jordan elimination with partial
// pivoting on the device (in place: one pivot kernel and one elimination kernel per column, then
// the column interchanges undone), and every coarse solve is one dense float64 matrix-vector
// product: gather the right-hand side, y = M^{-1} F, scatter y into (u, p).
#include <algorithm>
#include <cmath>

#include "cellops.cuh"
#include "kernels.cuh"

namespace smg {
namespace {

constexpr int kPivT = 1024;

// column k: pivot row p = argmax_{i >= k} |M[i][k]| (first of equal magnitudes), rows k and p
// swapped, row k scaled by 1 / M[k][k] with M[k][k] <- 1 / M[k][k], and the multipliers
// col[i] = M[i][k] (i != k) saved for the elimination.  A zero pivot sets *status.
__global__ void __launch_bounds__(kPivT) k_gj_pivot(double* __restrict__ M, int nb, int k, int* __restrict__ perm,
                                                     double* __restrict__ col, int* __restrict__ status) {
    __shared__ double sv[kPivT / 32];
    __shared__ int si[kPivT / 32];
    __shared__ int sp;
    __shared__ double sd;
    double best = -1.0;
    int bi = nb;
    for (int i = k + threadIdx.x; i < nb; i += kPivT) {
        const double v = fabs(M[(size_t)i * nb + k]);
        if (v > best) {
            best = v;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sv[warp] = best;
        si[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = -1.0;
        int p = k;
        for (int w = 0; w < kPivT / 32; ++w)
            if (sv[w] > b || (sv[w] == b && si[w] < p)) {
                b = sv[w];
                p = si[w];
            }
        if (p >= nb) p = k;
        sp = p;
        perm[k] = p;
    }
    __syncthreads();
    const int p = sp;
    if (p != k)
        for (int j = threadIdx.x; j < nb; j += kPivT) {
            const double t = M[(size_t)k * nb + j];
            M[(size_t)k * nb + j] = M[(size_t)p * nb + j];
            M[(size_t)p * nb + j] = t;
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d = M[(size_t)k * nb + k];
        if (!(fabs(d) > 1e-300)) {
            *status = 1;
            d = 1.0;
        }
        sd = d;
    }
    __syncthreads();
    const double inv_d = 1.0 / sd;
    for (int i = threadIdx.x; i < nb; i += kPivT) col[i] = i == k ? 0.0 : M[(size_t)i * nb + k];
    for (int j = threadIdx.x; j < nb; j += kPivT)
        M[(size_t)k * nb + j] = j == k ? inv_d : M[(size_t)k * nb + j] * inv_d;
}

// rows i != k: M[i][j] -= col[i] M[k][j] (j != k), M[i][k] = -col[i] M[k][k]
__global__ void __launch_bounds__(256) k_gj_elim(double* __restrict__ M, int nb, int k, const double* __restrict__ col) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= nb || i == k) return;
    const double c = col[i];
    if (c == 0.0) return;
    const double rk = M[(size_t)k * nb + j];
    if (j == k) M[(size_t)i * nb + k] = -c * rk;
    else M[(size_t)i * nb + j] -= c * rk;
}

// undo the row interchanges as column interchanges, last first (one thread per row)
__global__ void k_gj_unscramble(double* __restrict__ M, int nb, const int* __restrict__ perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double* r = M + (size_t)i * nb;
    for (int k = nb - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k) {
            const double t = r[k];
            r[k] = r[p];
            r[p] = t;
        }
    }
}

// (u, p) of the level with N = n = M^{-1} F, F = (f at the interior nodes, g): each warp forms one
// row's dot product with F (float64, F staged in shared memory), lane 0 stores the result.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_solve(int n, const double* __restrict__ inv, int nb,
                                                     const T* __restrict__ f, const T* __restrict__ g,
                                                     T* __restrict__ u, T* __restrict__ p) {
    pdl_wait();
    extern __shared__ double sF[];
    const int nm = 2 * n - 1, nv = nm * nm, nunk = nb - 1;
    const int ld = 2 * n + 1, n2 = ld * ld;
    for (int t = threadIdx.x; t < nunk; t += blockDim.x) {
        double v;
        if (t < 2 * nv) {
            const int c = t / nv, r = t - c * nv;
            const int X = r % nm + 1, Y = r / nm + 1;
            v = (double)f[c * n2 + Y * ld + X];
        } else {
            v = (double)g[t - 2 * nv];
        }
        sF[t] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < nunk; row += nwarps) {
        const double* r = inv + (size_t)row * nb;
        double acc = 0.0;
        for (int j = lane; j < nunk; j += 32) acc = fma(r[j], sF[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            if (row < 2 * nv) {
                const int c = row / nv, q = row - c * nv;
                u[c * n2 + (q / nm + 1) * ld + q % nm + 1] = (T)acc;
            } else {
                p[row - 2 * nv] = (T)acc;
            }
        }
    }
    pdl_trigger();
}

}  // namespace

// In-place inverse of the row-major nb x nb matrix M (device); perm (nb ints), col (nb doubles) and
// status (one int) are device scratch.  Asynchronous on s; *status != 0 afterwards means a zero
// pivot (singular matrix).
cudaError_t launch_dense_inverse(cudaStream_t s, double* M, int nb, int* perm, double* col, int* status) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const dim3 eg((nb + 255) / 256, nb);
    for (int k = 0; k < nb; ++k) {
        k_gj_pivot<<<1, kPivT, 0, s>>>(M, nb, k, perm, col, status);
        k_gj_elim<<<eg, 256, 0, s>>>(M, nb, k, col);
    }
    k_gj_unscramble<<<(nb + 127) / 128, 128, 0, s>>>(M, nb, perm);
    return cudaGetLastError();
}

template <typename T>
void launch_dense_solve(cudaStream_t s, int n, const double* inv, int nb, const T* f, const T* g, T* u, T* p) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int rows_per_cta = 8;
    const int grid = std::max(1, std::min(2 * std::max(sms, 1), (nb - 1 + rows_per_cta - 1) / rows_per_cta));
    launch_pdl(k_dense_solve<T>, dim3(grid), dim3(256), sizeof(double) * (size_t)(nb - 1), s, n, inv, nb, f, g, u, p);
}
template void launch_dense_solve<float>(cudaStream_t, int, const double*, int, const float*, const float*, float*,
                                        float*);
template void launch_dense_solve<double>(cudaStream_t, int, const double*, int, const double*, const double*,
                                         double*, double*);

cudaError_t prepare_dense_solve(int nb_max) {
    const int bytes = (int)(sizeof(double) * (size_t)(nb_max - 1));
    cudaError_t e = cudaFuncSetAttribute(k_dense_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dense_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

}  // namespace smg
