// timestep.cu -- right-hand side of one implicit Euler step of the time-dependent Stokes problem.
//
// Sec. 1: the generalized Stokes system arises in implicit time stepping, with beta proportional
// to the inverse time step.  For u_t - Laplace u + grad p = f, div u = g and the implicit Euler
// method with step dt, one step solves -Laplace u' + beta u' + grad p' = f' + beta u, div u' = g',
// beta = 1/dt.  The velocity load is linear in the nodal data, (f_h + beta u, phi_i), so the step's
// right-hand side is the load vector of the nodal values f' + beta u: this file forms those values
// and the load kernel applies the mass matrices.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>

namespace smg {

// w = f + beta u over n lattice values (both velocity components, boundary points included).
__global__ void k_euler_nodal(size_t n, double beta, const double* __restrict__ f,
                              const double* __restrict__ u, double* __restrict__ w) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        w[i] = f[i] + beta * u[i];
}

cudaError_t launch_euler_nodal(cudaStream_t st, size_t n, double beta, const double* f, const double* u,
                               double* w) {
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nt = 256;
    const size_t blocks = std::min<size_t>((n + nt - 1) / nt, (size_t)std::max(sms, 1) * 8);
    k_euler_nodal<<<(unsigned)blocks, nt, 0, st>>>(n, beta, f, u, w);
    return cudaGetLastError();
}

}  // namespace smg
