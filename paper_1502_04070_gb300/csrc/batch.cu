// batch.cu -- device-side loop control of the batched solver.
//
// Every instance of a batch runs its refinement steps inside a conditional WHILE node of one CUDA
// graph; after each step this kernel decides on the device whether the instance goes on, so the
// whole batch runs to convergence in one graph launch without returning to the host.
#include <cuda_runtime.h>

#include "cellops.cuh"
#include "kernels.cuh"

namespace smg {

// scal[0] = ||r||^2 of the last step, scal[2] = ||F||^2.  Continue while ||r||^2 > tol2 ||F||^2,
// the step count is below max_cycles and the residual is finite.
__global__ void k_batch_check(cudaGraphConditionalHandle hnd, const double* __restrict__ scal, double tol2,
                              int max_cycles, int* __restrict__ count) {
    pdl_wait();
    if (threadIdx.x != 0) return;
    const int c = *count + 1;
    *count = c;
    const double r2 = scal[0];
    const bool go = isfinite(r2) && r2 > tol2 * scal[2] && c < max_cycles;
    cudaGraphSetConditional(hnd, go ? 1u : 0u);
    pdl_trigger();
}

__global__ void k_batch_store(const double* __restrict__ scal, const int* __restrict__ count,
                              double* __restrict__ out) {
    pdl_wait();
    if (threadIdx.x != 0) return;
    out[0] = scal[0];
    out[1] = scal[2];
    out[2] = (double)*count;
    pdl_trigger();
}

// Single solves: the same device-side loop, with a residual history and a divergence test.
// ctl: [0] threshold factor (stop when r^2 <= ctl[0] * ||F||^2), [1] max steps, [2] previous r^2;
// ictl: [0] step count, [1] consecutive growths.  hist[c] = r^2 after step c (c < cap).
__global__ void k_solve_check(cudaGraphConditionalHandle hnd, const double* __restrict__ scal,
                              double* __restrict__ ctl, int* __restrict__ ictl, double* __restrict__ hist, int cap) {
    pdl_wait();
    if (threadIdx.x != 0) return;
    const int c = ictl[0] + 1;
    ictl[0] = c;
    const double r2 = scal[0];
    if (c < cap) hist[c] = r2;
    const int grow = r2 > ctl[2] ? ictl[1] + 1 : 0;
    ictl[1] = grow;
    ctl[2] = r2;
    const bool go = isfinite(r2) && r2 > ctl[0] * scal[2] && c < (int)ctl[1] && grow < 8;
    cudaGraphSetConditional(hnd, go ? 1u : 0u);
    pdl_trigger();
}

void launch_solve_check(cudaStream_t s, cudaGraphConditionalHandle hnd, const double* scal, double* ctl, int* ictl,
                        double* hist, int cap) {
    launch_pdl(k_solve_check, 1, 32, 0, s, hnd, scal, ctl, ictl, hist, cap);
}

void launch_batch_check(cudaStream_t s, cudaGraphConditionalHandle hnd, const double* scal, double tol2,
                        int max_cycles, int* count) {
    launch_pdl(k_batch_check, 1, 32, 0, s, hnd, scal, tol2, max_cycles, count);
}

void launch_batch_store(cudaStream_t s, const double* scal, const int* count, double* out) {
    launch_pdl(k_batch_store, 1, 32, 0, s, scal, count, out);
}

}  // namespace smg
