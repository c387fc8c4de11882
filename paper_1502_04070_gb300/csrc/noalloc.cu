// noalloc.cu -- residual norm for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that works inside a fixed memory budget handed out by
// another framework (an arena that owns the rest of the device), code on a device that is already
// full, or embedding code with no way to release memory later.  For them this file offers
// stokes_residual_norm2_noalloc(), a handle-free variant of the residual kernel whose only scratch
// (the per-block partial sums of the norm) lives in a file-scope __device__ array of fixed size.
// Each GPU that loads the library keeps that array (about 131 KB) until the process exits.
#include <cmath>
#include <mutex>

#include "../../include/stokes_mg.h"
#include "cellops.cuh"
#include "coef.h"
#include "kernels.cuh"

namespace smg {
namespace {

constexpr int kNoAllocMaxLevels = 11;   // finest level k <= 10, N <= 2048
constexpr int kNoAllocMaxN = 1 << kNoAllocMaxLevels;
constexpr int kNoAllocPartials = ((kNoAllocMaxN + 1 + BX - 1) / BX) * ((kNoAllocMaxN + 1 + BY - 1) / BY);

// Shared by every call on a device; see the thread-safety note in include/stokes_mg.h.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};          // device address of the array, per device (set-up once)

// ||F - A x||^2 partial sums per block: the residual kernel without its output arrays
__global__ void __launch_bounds__(NT) k_residual_sumsq(int n, const __grid_constant__ OpCoef<double> c,
                                                       const double* __restrict__ u, const double* __restrict__ p,
                                                       const double* __restrict__ f, const double* __restrict__ g,
                                                       double* __restrict__ partial) {
    CELL_INDEX
    const size_t n2 = (size_t)(2 * n + 1) * (2 * n + 1);
    double ss = 0.0;
    if (active) {
        Acc<double> a;
        cell_apply<true, true, true, false, true>(i, j, n, c.A, c, gview(u, 2 * n + 1), gview(u + n2, 2 * n + 1),
                                                  gview(p, n + 1), a);
        const CellNodes cn = cell_nodes(i, j, n);
        const int ld = 2 * n + 1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (!slot_unknown(cn, s)) continue;
            int X, Y;
            slot_pos(i, j, s, X, Y);
            const size_t idx = (size_t)Y * ld + X;
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
                const double r = f[comp * n2 + idx] - a.au[comp][s] - a.bt[comp][s];
                ss += r * r;
            }
        }
        const double r = g[(size_t)j * (n + 1) + i] - a.bu;
        ss += r * r;
    }
    const double t = block_sum2d(ss, tid);
    if (tid == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

}  // namespace
}  // namespace smg

using namespace smg;

extern "C" stokes_status stokes_residual_norm2_noalloc(int levels, double beta, const double* u, const double* p,
                                                       const double* f, const double* g, double* norm2,
                                                       void* stream) {
    if (levels < 1 || levels > kNoAllocMaxLevels || !(beta >= 0.0) || !std::isfinite(beta) || !u || !p || !f ||
        !g || !norm2)
        return STOKES_ERR_BAD_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return STOKES_ERR_CUDA;
    double* scratch = nullptr;
    {
        // set-up, once per device: the array's device address (host code cannot use the symbol itself)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess) return STOKES_ERR_CUDA;
            g_noalloc_ptr[dev] = static_cast<double*>(ptr);
        }
        scratch = g_noalloc_ptr[dev];
    }
    const int n = 1 << levels;
    const OpCoef<double> c = make_coef<double>(n, beta);
    cudaStream_t s = (cudaStream_t)stream;
    // each launch reports its own status (cudaLaunchKernelEx), so an error that the caller's earlier
    // work left pending in the runtime is neither blamed on this call nor cleared by it
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = cells_grid(n);
    cfg.blockDim = dim3(BX, BY);
    cfg.stream = s;
    if (cudaLaunchKernelEx(&cfg, k_residual_sumsq, n, c, u, p, f, g, scratch) != cudaSuccess) return STOKES_ERR_CUDA;
    if (launch_reduce(s, scratch, cells_blocks(n), norm2) != cudaSuccess) return STOKES_ERR_CUDA;
    return STOKES_OK;
}
