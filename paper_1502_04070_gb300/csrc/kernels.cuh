// kernels.cuh -- launch wrappers of the solver's CUDA kernels (defined in kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace smg {

// Partial-sum buffer capacity (blocks of the largest level) is computed by the caller with
// cells_blocks(n).
int cells_blocks(int n);

// Transfer weight table (constant memory), set once per device.
cudaError_t upload_transfer_weights(const double* P2 /* [2][9][5][5] */);

// r = F - A x with per-block partial sums of r.r (over unknowns) in `partial` (may be null) and an
// optional float32 copy of r in (ru2, rp2).
// dom: kDomSquare or kDomL (common.cuh: on the L, the nodes outside it are not unknowns)
template <typename T, typename TO>
void launch_residual(cudaStream_t s, int n, const OpCoef<T>& c, const T* u, const T* p, const T* f,
                     const T* g, TO* ru, TO* rp, double* partial, float* ru2 = nullptr, float* rp2 = nullptr,
                     int dom = kDomSquare);


// Uzawa step (Sec. 4), three kernels:
//   uh = u + tau Ahat^{-1} (f - A u - B^T p)
//   dp = sigma Shat^{-1} (B uh - g);  p += dp
//   u  = uh - tau Ahat^{-1} B^T dp
template <typename T>
void launch_uzawa(cudaStream_t s, int n, const OpCoef<T>& c, T tau, T sigma, T* u, T* p, const T* f,
                  const T* g, const T* sinv, T* uh, T* dp, int bx = 32, int by = 8, int dom = kDomSquare);

// Refinement update (see refine.cu): float32 correction e, float64 iterate x, residual r stored as
// (hi, lo) float pairs in the 8-byte slots of a float64 array:
//   x += e,  r -= A e  (error-free float32 products, ~2^-48 relative),  r32 = float(r),
//   partial sums of r.r; planar: e and r32 in the planar float32 layout (common.cuh); dom = kDomL:
//   the L's unknowns and pressure-mean weights (the nodes outside it keep zero).
void launch_ir_update_df(cudaStream_t s, int n, const OpCoef<float>& chi, const OpCoef<float>& clo,
                         const float* eu, const float* ep, double* xu, double* xp, double* ru, double* rp,
                         float* r32u, float* r32p, double* partial, double* wpartial, bool planar = false,
                         int dom = kDomSquare);
// p -= *scalar on every vertex (the zero-mean projection once the integral of p is reduced); on the
// L (dom = kDomL) p -= *scalar / (3/4) at the L's vertices
template <typename T>
void launch_psub(cudaStream_t s, int n, T* p, const double* scalar, int dom = kDomSquare);
void launch_residual_df(cudaStream_t s, int n, const OpCoef<double>& c, const double* u, const double* p,
                        const double* f, const double* g, double* ru, double* rp, float* r32u, float* r32p,
                        double* partial, bool planar = false,   // planar: (r32u, r32p) in the planar layout
                        int dom = kDomSquare);                   // kDomL: the L's unknowns only

// The same Uzawa step fused into one kernel with shared-memory halos: reads (u, p), writes
// (u_out, p_out) (distinct buffers).
template <typename T>
cudaError_t prepare_uzawa_fused();   // raises the kernel's shared-memory limit on the current device
// The float32 step on component-pair tiles with packed FP32x2 arithmetic (uzawa_pair.cu), 28 cells
// wide; variant 0: 8 warps, 1: 4 warps (tile height chosen per level), 2: 12 warps, 8 rows.  Reads
// (u, p), writes (u_out, p_out).
void launch_uzawa_pair(int variant, cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma,
                       const float* u, const float* p, const float* f, const float* g, const float* sinv,
                       float* u_out, float* p_out);
cudaError_t prepare_uzawa_pair();
// The float32 step with the operator's coefficients in registers and asynchronous staging
// (uzawa_reg.cu), 28 cells wide, 8 warps; variant 0: tile height for at least 2 CTAs per SM, 1: for at
// least 4.  Returns false (and launches
// nothing) if the level's coefficients do not have the compile-time structure the kernel assumes.
bool launch_uzawa_reg(int variant, cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma,
                      const float* u, const float* p, const float* f, const float* g, const float* sinv,
                      float* u_out, float* p_out);
cudaError_t prepare_uzawa_reg();
// The same step on a float32 level in the planar layout (common.cuh), its tiles staged by
// tensor-memory-access box copies; false (nothing launched) if the coefficients lack the register
// tile's structure or the driver offers no tensor-map encoder.  uzawa_tma_available: the encoder is
// there.  uzawa_tma_timeouts: nonzero if a CTA of the kernel gave up waiting (about a second) for
// its tiles since the last call; clears the flag (synchronises with the device).
constexpr int kDefaultTmaLevel = 6;   // lowest level held planar unless stokes_params.tma_level says otherwise
// With u given, the step starts from x + P x_c, x_c = (u, p) the iterate of the coarse level N / 2
// (planar or compact): the coarse-grid correction of Sec. 3 added to the staged tiles in shared
// memory (the separate prolongation kernel and its pass over the fine state are saved).
struct CoarseCorrection {
    const float* u = nullptr;
    const float* p = nullptr;
    bool planar = false;
};
bool launch_uzawa_tma(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, const float* u,
                      const float* p, const float* f, const float* g, const float* sinv, float* u_out, float* p_out,
                      const CoarseCorrection& cc = CoarseCorrection{});
bool uzawa_tma_available();
// the fused correction can be used: the tensor-map encoder is there and the kernel's compile-time
// embedding table equals the host element code's transfer weights
bool uzawa_tma_embed_available();
// that compile-time table, w[((o * 9 + L) * 4 + fb) * 4 + fa] (host only)
void embed_weights_table(double* w);
// false when the environment sets STOKES_MG_FUSE_PROLONG=0 (read once per process): the planar
// levels then prolongate with the separate kernel
bool fuse_prolong_enabled();
// Variants of the planar step, one tile per CTA of 8 warps: 0 tile height for 3 CTAs per SM (80
// registers), 2 for 4 CTAs per SM (64 registers); 1, 3 the same, each CTA also prefetching into L2
// the tiles of the tile one wave of resident CTAs ahead; 4, 5 two rows per warp pass (the shared
// window rows loaded once; even tile heights), 2 or 3 CTAs per SM, with the prefetch.
// launch_uzawa_tma runs the variant chosen for level size n (0 until autotune_uzawa_tma or
// set_tma_choice).
constexpr int kTmaVariants = 6;
bool launch_uzawa_tma_variant(int variant, cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma,
                              const float* u, const float* p, const float* f, const float* g, const float* sinv,
                              float* u_out, float* p_out, const CoarseCorrection& cc = CoarseCorrection{});
// r = F - A x on a planar level (N = n) and its restriction (fc, gc) = I^T r to the coarse level
// (planar or not: pc_planar), with the coarse iterate (uc, pc) set to zero, in one kernel on the
// tiles of the planar step; the fine defect stays in shared memory.  False (nothing launched) as
// for launch_uzawa_tma.
bool launch_restrict_tma(cudaStream_t s, int n, bool pc_planar, const OpCoef<float>& c, const float* u, const float* p,
                         const float* f, const float* g, float* fc, float* gc, float* uc, float* pc);
// The float32 V- or W-cycle from level `top` (compact layout, top <= kSmallCycleTop) down to the
// coarsest level clev of the iteration, with its exact solve, in ONE cooperative launch (uzawa_reg.cu):
// every CTA resident, phases separated by grid barriers whose waits are bounded (about a second; a
// timeout sets the flag uzawa_tma_timeouts() reports).  On entry (u, p) of `top` hold its iterate and
// (f, g) its right-hand side; on exit (u, p) hold the iterate after the cycle.  Arrays per level
// (index = level, N = 2^(level + 1)); coef_host: the levels' operators (host), coef_dev: the same on the
// device; inv0: the level-0 bordered inverse (clev = 0), cinv / cnb: the level-clev one (clev > 0);
// bar: one device word, cleared by the launch (stream-ordered) and used by the barriers.
constexpr int kSmallCycleTop = 6;
struct SmallCycleHost {
    float *u[kSmallCycleTop + 1], *p[kSmallCycleTop + 1], *f[kSmallCycleTop + 1], *g[kSmallCycleTop + 1];
    float *tu[kSmallCycleTop + 1], *tp[kSmallCycleTop + 1];
    const float* sinv[kSmallCycleTop + 1];
    const OpCoef<float>* coef_host[kSmallCycleTop + 1];
    const OpCoef<float>* coef_dev;
    const double* inv0;
    const double* cinv;
    int cnb;
    unsigned* bar;
    float tau, sigma;
    int nu_pre, nu_post, gamma, top, clev;
};
cudaError_t launch_small_cycle(cudaStream_t s, const SmallCycleHost& h);
int tma_choice(int n);
bool tma_tuned(int n);
bool set_tma_choice(int n, int v);
// times every planar variant on these planar buffers (contents overwritten) and keeps the fastest
cudaError_t autotune_uzawa_tma(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, float* u,
                               float* p, const float* f, const float* g, const float* sinv, float* u_out, float* p_out);
unsigned uzawa_tma_timeouts();
// Does the compile-time structure of the register tile match these coefficients?
bool reg_tables_match(const OpCoef<float>& c);
template <typename T>
cudaError_t launch_uzawa_fused(cudaStream_t s, int n, const OpCoef<T>& c, T tau, T sigma, const T* u, const T* p,
                               const T* f, const T* g, const T* sinv, T* u_out, T* p_out);
// One float32 Uzawa step with the variant the autotuner chose for level size n: either a fused
// one-kernel step from (u, p) into (u_out, p_out) (returns true), or the three-kernel step in place
// on (u, p) with (u_out, p_out) as scratch (returns false).
bool uzawa_tuned(int n);
int uzawa_choice(int n);
bool set_uzawa_choice(int n, int v);   // false if v is not a step variant
bool launch_uzawa_auto(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, float* u, float* p,
                       const float* f, const float* g, const float* sinv, float* u_out, float* p_out);
// Picks the fastest float32 tile shape for level size n by timing each on these buffers (their
// contents are overwritten); returns the variant index and its time per step.
cudaError_t autotune_uzawa_fused(cudaStream_t s, int n, const OpCoef<float>& c, float tau, float sigma, float* u,
                                 float* p, const float* f, const float* g, const float* sinv, float* u_out,
                                 float* p_out, int* chosen, float* best_ms);

// Normal-equation step (Sec. 4): x += tau L^{-1} A L^{-1} (F - A x),  L = diag(Ahat, Shat).
template <typename T>
void launch_normal_eq(cudaStream_t s, int n, const OpCoef<T>& c, T tau, T* u, T* p, const T* f,
                      const T* g, const T* sinv, T* zu, T* zp);

// (fc, gc) = I^T (ru, rp): fine level n = 2 nc.
template <typename T>
void launch_restrict(cudaStream_t s, int nc, const T* ru, const T* rp, T* fc, T* gc, T* uc = nullptr,
                     T* pc = nullptr, int dom = kDomSquare);   // uc, pc: optional coarse iterate set to zero

// (u, p) += I (uc, pc)
template <typename T>
void launch_prolong_add(cudaStream_t s, int nc, const T* uc, const T* pc, T* u, T* p, int dom = kDomSquare);

// Float32 levels in the planar layout (common.cuh): the residual of a planar level, and the transfers
// between a planar fine level (N = 2 nc) and its coarse level, planar or not (pc_planar).
void launch_residual_planar(cudaStream_t s, int n, const OpCoef<float>& c, const float* u, const float* p,
                            const float* f, const float* g, float* ru, float* rp);
void launch_restrict_planar(cudaStream_t s, int nc, bool pc_planar, const float* ru, const float* rp, float* fc,
                            float* gc, float* uc, float* pc);
void launch_prolong_add_planar(cudaStream_t s, int nc, bool pc_planar, const float* uc, const float* pc, float* u,
                               float* p);
// compact <-> planar copies of a float32 level state (u: velocity, p: vertex array); to_planar writes
// zero at the boundary nodes and the padding of the planar velocity array
void launch_to_planar(cudaStream_t s, int n, const float* u, const float* p, float* pu, float* pp);
void launch_from_planar(cudaStream_t s, int n, const float* pu, const float* pp, float* u, float* p);

// level-0 exact solve with the bordered inverse (27 x 27, float64)
template <typename T>
void launch_coarse_solve(cudaStream_t s, const double* inv, const T* f, const T* g, T* u, T* p);

// The L-shaped domain: zero the entries outside the L (velocity: the closed removed quadrant; vertices:
// strictly inside it) of a float64 velocity array u and / or vertex array p (either may be null).
void launch_mask_l(cudaStream_t s, int n, double* u, double* p);

// Exact solve on a coarsest level c > 0 (dense.cu): in-place float64 inverse of the bordered
// system (row-major nb x nb, device; perm, col, status device scratch; *status != 0 = singular), and
// (u, p) = M^{-1} (f, g) on the level with N = n.
cudaError_t launch_dense_inverse(cudaStream_t s, double* M, int nb, int* perm, double* col, int* status);
template <typename T>
void launch_dense_solve(cudaStream_t s, int n, const double* inv, int nb, const T* f, const T* g, T* u, T* p);
cudaError_t prepare_dense_solve(int nb_max);
constexpr int kMaxCoarseLevel = 3;   // N = 16: a bordered system of 2212 unknowns

// Shat^{-1} per vertex (float64 computation, stored as T), rows of vld entries (0: N + 1)
template <typename T>
void launch_schur_diag(cudaStream_t s, int n, const OpCoef<double>& c, T* sinv, int dom = kDomSquare, int vld = 0);

// p <- p - sum_i w_i p_i  (w = M_P 1, sum w = 1): partial sums then subtraction
template <typename T>
void launch_pmean(cudaStream_t s, int n, T* p, double* partial, double* scalar, int dom = kDomSquare);

// out[0] = sum of partial[0..count); returns the launch's own status
cudaError_t launch_reduce(cudaStream_t s, const double* partial, int count, double* out);

// load vectors: f = M_U f_nodal (interior rows), g = M_P g_nodal, with optional zero-mean shift
template <typename T>
void launch_load(cudaStream_t s, int n, const MassCoef<T>& m, const T* fn, const T* gn, T* f, T* g,
                 int project_g, double* partial, double* scalar);

// partial sums of a^T M_U b
void launch_mass_dot(cudaStream_t s, int n, const MassCoef<double>& m, const double* a, const double* b,
                     double* partial);

// partial sums of ||F||^2 over the unknowns (f at interior velocity nodes, all of g)
void launch_rhs_norm(cudaStream_t s, int n, const double* f, const double* g, double* partial);

// g <- g - (1^T g) w  with w = M_P 1: the pressure right-hand side becomes orthogonal to the
// constant pressure (the kernel of the saddle-point matrix)
void launch_make_consistent(cudaStream_t s, int n, double* g, double* partial, double* scalar);

// The float32 V-cycle of levels 0..a.top (top <= 4) in one CTA with shared-memory arrays
// (coarse_cycle.cuh); the kernel's shared-memory limit is raised by prepare_coarse_cycle().
constexpr int kCoarseCycleTop = 4;
struct CoarseCycleArgs {
    OpCoef<float> c[kCoarseCycleTop];     // levels 1..top at index l - 1
    const float* sinv[kCoarseCycleTop];   // Shat^{-1} of levels 1..top (global)
    const double* inv;                    // level-0 bordered inverse (27 x 27, global)
    float* u;                             // iterate of level `top` (global; read at start, written at end)
    float* p;
    const float* f;                       // right-hand side of level `top` (global)
    const float* g;
    float tau, sigma;
    int nu_pre, nu_post;
    int top;                              // 1 <= top <= kCoarseCycleTop
};
// kernel parameters are limited to 32,764 bytes
static_assert(sizeof(CoarseCycleArgs) <= 32764, "coarse-cycle parameters exceed the launch limit");

cudaError_t prepare_coarse_cycle();
void launch_coarse_cycle(cudaStream_t s, const CoarseCycleArgs& a);

// batched solver: device-side WHILE condition and result store (batch.cu)
void launch_batch_check(cudaStream_t s, cudaGraphConditionalHandle hnd, const double* scal, double tol2,
                        int max_cycles, int* count);
void launch_batch_store(cudaStream_t s, const double* scal, const int* count, double* out);
void launch_solve_check(cudaStream_t s, cudaGraphConditionalHandle hnd, const double* scal, double* ctl, int* ictl,
                        double* hist, int cap);

// x64 += e32 (count elements), and float64 -> float32 conversion
void launch_add_f32(cudaStream_t s, size_t count, const float* e, double* x);

}  // namespace smg
