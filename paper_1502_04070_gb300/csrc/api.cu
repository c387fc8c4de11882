// api.cu -- the C-ABI of include/stokes_mg.h: level hierarchy, cycle orchestration, solve loop.
//
// The multigrid iteration is the one of Sec. 3: nu_pre smoothing steps, restriction of the defect
// with the transposed embedding, gamma recursive iterations on the coarser level from zero (an exact
// solve on level 0), prolongation and correction, nu_post smoothing steps.  The whole iteration,
// the zero-mean pressure projection and the residual norm are captured once into a CUDA graph and
// replayed per cycle; the host reads one scalar per cycle to test convergence.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/stokes_mg.h"
#include "coef.h"
#include "elements.h"
#include "kernels.cuh"

namespace smg {
// timestep.cu: w = f + beta u over n values (the nodal data of an implicit Euler right-hand side)
cudaError_t launch_euler_nodal(cudaStream_t st, size_t n, double beta, const double* f, const double* u, double* w);
}  // namespace smg

using namespace smg;

namespace {

// A named range around each public call that launches work, for timeline profilers (NVTX: header-only,
// no cost unless a profiler is attached).
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
};

}  // namespace

namespace {

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return fail(e_);    \
    } while (0)

stokes_status fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return STOKES_ERR_OOM;
    }
    return STOKES_ERR_CUDA;
}

// Device memory of a handle or batch: through the allocator registered with stokes_set_allocator
// when the handle was set up, else cudaMalloc / cudaFree.  Keeps the size of every live block (the
// release callback receives it).
struct DevMem {
    stokes_alloc_fn alloc = nullptr;
    stokes_free_fn release = nullptr;
    void* ctx = nullptr;
    cudaStream_t st = nullptr;
    std::vector<std::pair<void*, size_t>> live;
    cudaError_t get(void** p, size_t bytes) {
        *p = nullptr;
        if (alloc) {
            *p = alloc(bytes, (void*)st, ctx);
            if (!*p) return cudaErrorMemoryAllocation;
        } else {
            cudaError_t e = cudaMalloc(p, bytes);
            if (e != cudaSuccess) return e;
        }
        live.emplace_back(*p, bytes);
        return cudaSuccess;
    }
    template <typename T>
    cudaError_t get(T** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = get(&q, bytes);
        *p = static_cast<T*>(q);
        return e;
    }
    void put(void* p) {
        if (!p) return;
        for (size_t i = 0; i < live.size(); ++i)
            if (live[i].first == p) {
                if (release) release(p, live[i].second, (void*)st, ctx);
                else cudaFree(p);
                live[i] = live.back();
                live.pop_back();
                return;
            }
    }
    void put_all() {
        while (!live.empty()) put(live.back().first);
    }
};

std::mutex g_alloc_mu;
stokes_alloc_fn g_alloc = nullptr;
stokes_free_fn g_release = nullptr;
void* g_alloc_ctx = nullptr;

void init_mem(DevMem& m, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    m.alloc = g_alloc;
    m.release = g_release;
    m.ctx = g_alloc_ctx;
    m.st = st;
}

template <typename T>
struct Level {
    int n = 0;
    size_t n2 = 0, n1 = 0;   // (2n+1)^2 and (n+1)^2; planar: half the velocity array and the vertex array
    bool planar = false;     // float32 level in the planar layout (common.cuh), smoothed by the TMA step
    T *u = nullptr, *p = nullptr, *f = nullptr, *g = nullptr;
    T *tu = nullptr, *tp = nullptr, *sinv = nullptr;
    void* slab = nullptr;
    OpCoef<T> c{};
};

template <typename T>
stokes_status alloc_level(Level<T>& L, int k, DevMem& mem, bool planar = false) {
    L.n = 1 << (k + 1);
    L.planar = planar;
    L.n2 = planar ? pl_ucount(L.n) / 2 : (size_t)(2 * L.n + 1) * (2 * L.n + 1);
    L.n1 = planar ? pl_pcount(L.n) : (size_t)(L.n + 1) * (L.n + 1);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t bu = al(2 * L.n2 * sizeof(T)), bp = al(L.n1 * sizeof(T));
    const size_t total = 3 * bu + 4 * bp;
    CK(mem.get(&L.slab, total));
    char* q = (char*)L.slab;
    L.u = (T*)q; q += bu;
    L.f = (T*)q; q += bu;
    L.tu = (T*)q; q += bu;
    L.p = (T*)q; q += bp;
    L.g = (T*)q; q += bp;
    L.tp = (T*)q; q += bp;
    L.sinv = (T*)q;
    CK(cudaMemsetAsync(L.slab, 0, total, mem.st));
    return STOKES_OK;
}

std::mutex g_dev_mu;
unsigned long long g_dev_weights = 0;   // devices whose constant transfer table is set

stokes_status ensure_weights() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (dev < 64 && (g_dev_weights >> dev) & 1ull) return STOKES_OK;
    static TransferWeights W = transfer_weights();
    CK(upload_transfer_weights(&W.P2[0][0][0][0]));
    if (dev < 64) g_dev_weights |= 1ull << dev;
    return STOKES_OK;
}

}  // namespace

struct stokes_handle_t {
    stokes_params prm{};
    cudaStream_t st = nullptr;
    DevMem mem;                             // every device buffer of the handle
    bool own_stream = false;
    int L = 0;                              // number of levels
    std::vector<Level<double>> h64;         // FP64: all levels; MIXED: finest only
    std::vector<Level<float>> h32;          // MIXED: all levels
    double* inv = nullptr;                  // level-0 bordered inverse (27 x 27)
    int dom = kDomSquare;                   // the domain: kDomSquare, or kDomL (common.cuh)
    int clev = 0;                           // coarsest level of the iteration (exact solve there)
    int cnb = 0;                            // clev > 0: size of its bordered system
    double* cinv = nullptr;                 // clev > 0: its inverse, cnb x cnb, float64
    int* cperm = nullptr;                   // clev > 0: scratch of the inversion
    double* ccol = nullptr;
    int* cstat = nullptr;
    double* partial = nullptr;
    int npartial = 0;
    double* scal = nullptr;                 // device scalars
    double* hscal = nullptr;                // pinned host mirror
    MassCoef<double> mass{};
    OpCoef<float> chi{}, clo{};             // MIXED: finest float64 coefficients split hi + lo
    bool coarse_kernel = true;              // float32 levels <= 4 in one shared-memory kernel
    bool launch_failed = false;             // a step variant refused to launch (reported by the next call)
    bool has_planar = false;                // some float32 level is planar
    int small_top = -1;                     // float32 levels clev+1..small_top: one cooperative launch per visit
    bool fuse_prolong = false;              // planar levels: x += P x_c inside the first post-smoothing step
    OpCoef<float>* dcoef = nullptr;         // device copies of the float32 operators of levels 0..small_top
    unsigned* dbar = nullptr;               // grid-barrier counter of that launch
    cudaGraphExec_t step = nullptr;         // one cycle + projection + residual norm
    int step_kernels = 0;                   // kernel nodes in `step`
    cudaGraphExec_t loop = nullptr;         // WHILE(not converged) { step; device-side test }
    int loop_kernels = 0;                   // kernels per loop iteration
    double* dctl = nullptr;                 // loop control (see k_solve_check), device
    int* ictl = nullptr;
    double* dhist = nullptr;                // residual^2 per step, device (kHistCap entries)
    double* hhist = nullptr;                // pinned mirror
    double* euler_w = nullptr;              // nodal data of an implicit Euler right-hand side
    cudaGraphExec_t euler = nullptr;        // a sequence of implicit Euler steps (stokes_euler_run)
    std::vector<const void*> euler_key;     // pointers (and so steps) it was built for
    double euler_tol = -1.0;                // tol and max_cycles it was built for
    int euler_max = -1;
    int* d_ecount = nullptr;                // device: cycles per step
    double* d_eres = nullptr;               // device: per step (true ||r||^2, ||F||^2, cycles)
    int euler_kernels = 0, euler_body = 0;  // kernels outside / inside the loop bodies
    unsigned long long launches = 0;        // kernels launched by this handle (graph nodes included)
    // optional timing of the finest-level smoothing steps and of the float64 residual: event
    // pairs recorded inside the captured graph (cudaEventRecordExternal)
    bool timing = false;
    std::vector<cudaEvent_t> ev;            // pairs: [2i] start, [2i+1] end
    int ev_smooth = 0, ev_resid = 0;        // pairs used by one graph launch
    int ev_cursor = 0;                      // pair index while capturing
    std::vector<unsigned char> ev_kind;     // per pair: kEvSmooth, kEvFused or kEvResid
    double t_smooth = 0.0, t_resid = 0.0;   // accumulated milliseconds
    long long n_smooth = 0, n_resid = 0;    // accumulated launches (groups)
    double t_fused = 0.0;                   // smoothing steps that also add the coarse-grid correction
    long long n_fused = 0;

    static constexpr int kHistCap = 4096;
    Level<double>& fin() { return h64.back(); }
    bool mixed() const { return prm.precision == STOKES_MIXED; }
};

namespace {

enum : unsigned char { kEvSmooth = 0, kEvFused = 1, kEvResid = 2 };
int ev_begin(stokes_handle* h, unsigned char kind) {
    if (!h->timing || h->ev_cursor * 2 + 1 >= (int)h->ev.size()) return -1;
    const int k = h->ev_cursor++;
    h->ev_kind[k] = kind;
    cudaEventRecordWithFlags(h->ev[2 * k], h->st, cudaEventRecordExternal);
    return k;
}
void ev_end(stokes_handle* h, int k) {
    if (k >= 0) cudaEventRecordWithFlags(h->ev[2 * k + 1], h->st, cudaEventRecordExternal);
}

// The status a call reports once its work is done: STOKES_ERR_CUDA if a step variant refused to
// launch (recorded while launching or capturing), STOKES_ERR_TIMEOUT if a CTA of the planar levels'
// step gave up waiting for its tiles (a device-wide flag, cleared by the read), else st.
stokes_status take_launch_failure(stokes_handle* h, stokes_status st = STOKES_OK) {
    if (h->launch_failed) {
        h->launch_failed = false;
        return STOKES_ERR_CUDA;
    }
    if (h->has_planar) {
        CK(cudaStreamSynchronize(h->st));
        if (uzawa_tma_timeouts()) return STOKES_ERR_TIMEOUT;
    }
    return st;
}

// nu smoothing steps on level lv.  The state is in (u, p) when `sw` is false and in (tu, tp)
// when true; returns where it is afterwards.  The fused float32 Uzawa kernel writes the other
// buffer pair (ping-pong); the float64 and normal-equation steps work in place and use the other
// pair as scratch.  With `coarse` given (a planar level), the first step adds the coarse-grid
// correction P x_c of that coarse level to its staged tiles before it smooths.
template <typename T>
bool smooth_level(stokes_handle* h, Level<T>& lv, int steps, bool timed, bool sw, const Level<T>* coarse = nullptr) {
    const stokes_params& P = h->prm;
    const bool f32 = sizeof(T) == 4 && P.smoother == STOKES_UZAWA;
    for (int s = 0; s < steps; ++s) {
        const bool fused = coarse && s == 0 && lv.planar;
        const int k = timed ? ev_begin(h, fused ? kEvFused : kEvSmooth) : -1;
        if (k >= 0) h->ev_smooth++;
        T* xu = sw ? lv.tu : lv.u;
        T* xp = sw ? lv.tp : lv.p;
        T* ou = sw ? lv.u : lv.tu;
        T* op = sw ? lv.p : lv.tp;
        if (P.smoother == STOKES_NORMAL_EQ) {
            launch_normal_eq<T>(h->st, lv.n, lv.c, (T)P.tau, xu, xp, lv.f, lv.g, lv.sinv, ou, op);
        } else if constexpr (sizeof(T) == 4) {
            if (h->dom == kDomL) {   // the L: the per-phase kernels (in place), the removed quadrant kept zero
                launch_uzawa<float>(h->st, lv.n, lv.c, (float)P.tau, (float)P.sigma, xu, xp, lv.f, lv.g, lv.sinv, ou, op,
                                    32, 8, h->dom);
            } else if (lv.planar) {
                CoarseCorrection cc;
                if (coarse && s == 0) cc = CoarseCorrection{coarse->u, coarse->p, coarse->planar};
                if (launch_uzawa_tma(h->st, lv.n, lv.c, (float)P.tau, (float)P.sigma, xu, xp, lv.f, lv.g, lv.sinv, ou,
                                     op, cc))
                    sw = !sw;
                else
                    h->launch_failed = true;
            } else if (f32 && launch_uzawa_auto(h->st, lv.n, lv.c, (float)P.tau, (float)P.sigma, xu, xp, lv.f, lv.g,
                                                lv.sinv, ou, op)) {
                sw = !sw;
            }
        } else {
            launch_uzawa<T>(h->st, lv.n, lv.c, (T)P.tau, (T)P.sigma, xu, xp, lv.f, lv.g, lv.sinv, ou, op, 32, 8, h->dom);
        }
        ev_end(h, k);
    }
    return sw;
}

// Sec. 3: one multigrid iteration on level l of hierarchy H (x = (u, p), F = (f, g) of the level);
// the iterate is in (u, p) on entry and on exit.
template <typename T>
void mg_cycle(stokes_handle* h, std::vector<Level<T>>& H, int l) {
    Level<T>& lv = H[l];
    if (l == h->clev) {   // the coarsest level of the iteration: exact solve (Sec. 3)
        if (l == 0) launch_coarse_solve<T>(h->st, h->inv, lv.f, lv.g, lv.u, lv.p);
        else launch_dense_solve<T>(h->st, lv.n, h->cinv, h->cnb, lv.f, lv.g, lv.u, lv.p);
        return;
    }
    if constexpr (sizeof(T) == 4) {
        // small levels: the whole V- or W-cycle from level l down in one cooperative launch
        if (l <= h->small_top && l > h->clev) {
            SmallCycleHost sh{};
            for (int k = h->clev; k <= l; ++k) {
                Level<float>& L = H[k];
                sh.u[k] = L.u;
                sh.p[k] = L.p;
                sh.f[k] = L.f;
                sh.g[k] = L.g;
                sh.tu[k] = L.tu;
                sh.tp[k] = L.tp;
                sh.sinv[k] = L.sinv;
                sh.coef_host[k] = &L.c;
            }
            sh.coef_dev = h->dcoef;
            sh.inv0 = h->inv;
            sh.cinv = h->cinv;
            sh.cnb = h->cnb;
            sh.bar = h->dbar;
            sh.tau = (float)h->prm.tau;
            sh.sigma = (float)h->prm.sigma;
            sh.nu_pre = h->prm.nu_pre;
            sh.nu_post = h->prm.nu_post;
            sh.gamma = h->prm.gamma;
            sh.top = l;
            sh.clev = h->clev;
            if (launch_small_cycle(h->st, sh) != cudaSuccess) h->launch_failed = true;
            return;
        }
        // small levels: the whole V-cycle from level l down in one CTA (shared memory)
        if (l <= kCoarseCycleTop && h->prm.gamma == 1 && h->prm.smoother == STOKES_UZAWA && h->coarse_kernel &&
            h->clev == 0) {
            CoarseCycleArgs a;
            for (int k = 1; k <= l; ++k) {
                a.c[k - 1] = H[k].c;
                a.sinv[k - 1] = H[k].sinv;
            }
            a.inv = h->inv;
            a.u = lv.u;
            a.p = lv.p;
            a.f = lv.f;
            a.g = lv.g;
            a.tau = (float)h->prm.tau;
            a.sigma = (float)h->prm.sigma;
            a.nu_pre = h->prm.nu_pre;
            a.nu_post = h->prm.nu_post;
            a.top = l;
            launch_coarse_cycle(h->st, a);
            return;
        }
    }
    const bool top = l == (int)H.size() - 1;
    bool sw = smooth_level(h, lv, h->prm.nu_pre, top, false);
    const Level<T>* fused_coarse = nullptr;   // the coarse-grid correction goes into the first post-smoothing step
    T* xu = sw ? lv.tu : lv.u;
    T* xp = sw ? lv.tp : lv.p;
    T* ru = sw ? lv.u : lv.tu;
    T* rp = sw ? lv.p : lv.tp;
    Level<T>& cl = H[l - 1];
    if constexpr (sizeof(T) == 4) {
        if (lv.planar) {
            // the defect and its restriction in one kernel on the staged tiles (the defect stays on chip)
            if (!launch_restrict_tma(h->st, lv.n, cl.planar, lv.c, xu, xp, lv.f, lv.g, cl.f, cl.g, cl.u, cl.p)) {
                launch_residual_planar(h->st, lv.n, lv.c, xu, xp, lv.f, lv.g, ru, rp);
                launch_restrict_planar(h->st, cl.n, cl.planar, ru, rp, cl.f, cl.g, cl.u, cl.p);
            }
            for (int r = 0; r < h->prm.gamma; ++r) mg_cycle(h, H, l - 1);
            if (h->fuse_prolong && h->prm.nu_post > 0) fused_coarse = &cl;
            else launch_prolong_add_planar(h->st, cl.n, cl.planar, cl.u, cl.p, xu, xp);
        }
    }
    if (!lv.planar) {
        launch_residual<T, T>(h->st, lv.n, lv.c, xu, xp, lv.f, lv.g, ru, rp, nullptr, nullptr, nullptr, h->dom);
        launch_restrict<T>(h->st, cl.n, ru, rp, cl.f, cl.g, cl.u, cl.p, h->dom);   // and the coarse iterate := 0
        for (int r = 0; r < h->prm.gamma; ++r) mg_cycle(h, H, l - 1);
        launch_prolong_add<T>(h->st, cl.n, cl.u, cl.p, xu, xp, h->dom);
    }
    sw = smooth_level(h, lv, h->prm.nu_post, top, sw, fused_coarse);
    if (sw) {   // odd number of ping-pong steps: bring the iterate back to (u, p)
        cudaMemcpyAsync(lv.u, lv.tu, 2 * lv.n2 * sizeof(T), cudaMemcpyDeviceToDevice, h->st);
        cudaMemcpyAsync(lv.p, lv.tp, lv.n1 * sizeof(T), cudaMemcpyDeviceToDevice, h->st);
    }
}

// True float64 residual of the finest state, its norm^2 into scal[0].  In MIXED mode the residual
// is kept in float64 (the finest temporaries) for the refinement updates and copied to float32 as
// the right-hand side of the next correction problem.
void residual_norm_fin(stokes_handle* h, bool timed = false) {
    Level<double>& F = h->fin();
    const int k = timed ? ev_begin(h, kEvResid) : -1;
    if (k >= 0) h->ev_resid++;
    if (h->mixed()) {
        // x in float64; r kept as two floats for the refinement updates, r32 = its float32 value
        Level<float>& E = h->h32.back();
        launch_residual_df(h->st, F.n, F.c, F.u, F.p, F.f, F.g, F.tu, F.tp, E.f, E.g, h->partial, E.planar, h->dom);
    } else {
        launch_residual<double, double>(h->st, F.n, F.c, F.u, F.p, F.f, F.g, F.tu, F.tp, h->partial, nullptr, nullptr,
                                        h->dom);
    }
    ev_end(h, k);
    launch_reduce(h->st, h->partial, cells_blocks(F.n), h->scal);
}

// One outer iteration on the internal finest state, ending with ||F - A x||^2 in scal[0].
void record_step(stokes_handle* h) {
    Level<double>& F = h->fin();
    if (h->mixed()) {
        Level<float>& E = h->h32.back();
        cudaMemsetAsync(E.u, 0, 2 * E.n2 * sizeof(float), h->st);
        cudaMemsetAsync(E.p, 0, E.n1 * sizeof(float), h->st);
        for (int c = 0; c < h->prm.inner_cycles; ++c) mg_cycle<float>(h, h->h32, h->L - 1);
        // x += e, r -= A e (two-float residual, error-free float32 products), r32 = float(r)
        const int k = ev_begin(h, kEvResid);
        if (k >= 0) h->ev_resid++;
        // the same pass leaves the partial sums of the zero-mean projection of x_p (second half)
        const int nb = cells_blocks(F.n);
        launch_ir_update_df(h->st, F.n, h->chi, h->clo, E.u, E.p, F.u, F.p, F.tu, F.tp, E.f, E.g, h->partial,
                            h->partial + nb, E.planar, h->dom);
        ev_end(h, k);
        launch_reduce(h->st, h->partial, nb, h->scal);
        launch_reduce(h->st, h->partial + nb, nb, h->scal + 1);
        launch_psub<double>(h->st, F.n, F.p, h->scal + 1, h->dom);
    } else {
        mg_cycle<double>(h, h->h64, h->L - 1);
        launch_pmean<double>(h->st, F.n, F.p, h->partial, h->scal + 1, h->dom);
        residual_norm_fin(h, true);
    }
}

stokes_status build_graph(stokes_handle* h) {
    if (h->step) return STOKES_OK;
    cudaGraph_t g = nullptr;
    h->ev_cursor = h->ev_smooth = h->ev_resid = 0;
    CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    record_step(h);
    cudaError_t e = cudaStreamEndCapture(h->st, &g);
    if (e != cudaSuccess) return fail(e);
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    h->step_kernels = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) h->step_kernels++;
    }
    e = cudaGraphInstantiate(&h->step, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->step = nullptr;
        return fail(e);
    }
    return STOKES_OK;
}

// The solve loop on the device: one conditional WHILE node whose body is one step followed by
// k_solve_check (convergence, step limit, divergence).  No event records (not allowed in bodies).
stokes_status build_loop(stokes_handle* h) {
    if (h->loop) return STOKES_OK;
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0));
    cudaError_t e;
    cudaGraphConditionalHandle hnd;
    cudaGraphNode_t nc;
    cudaGraphNodeParams cp = {};
    const bool timing = h->timing;
    h->timing = false;
    if ((e = cudaGraphConditionalHandleCreate(&hnd, top, 1, cudaGraphCondAssignDefault)) == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hnd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&nc, top, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            record_step(h);
            launch_solve_check(h->st, hnd, h->scal, h->dctl, h->ictl, h->dhist, stokes_handle_t::kHistCap);
            e = cudaStreamEndCapture(h->st, &body);
        }
        if (e == cudaSuccess) {
            size_t nn = 0;
            cudaGraphGetNodes(body, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(body, nodes.data(), &nn);
            h->loop_kernels = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) h->loop_kernels++;
            }
        }
    }
    h->timing = timing;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->loop, top, 0);
    cudaGraphDestroy(top);
    if (e != cudaSuccess) {
        h->loop = nullptr;
        return fail(e);
    }
    return STOKES_OK;
}

stokes_status launch_step(stokes_handle* h) {
    CK(cudaGraphLaunch(h->step, h->st));
    h->launches += h->step_kernels;
    return STOKES_OK;
}

// after the stream is synchronised: add the event intervals of the last graph launch
void collect_timing(stokes_handle* h) {
    if (!h->timing) return;
    for (int k = 0; k < h->ev_smooth + h->ev_resid; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (h->ev_kind[k] == kEvSmooth) {
            h->t_smooth += ms;
            h->n_smooth++;
        } else if (h->ev_kind[k] == kEvFused) {
            h->t_fused += ms;
            h->n_fused++;
        } else {
            h->t_resid += ms;
            h->n_resid++;
        }
    }
}

stokes_status rebuild_beta(stokes_handle* h) {
    const double beta = h->prm.beta;
    for (auto& lv : h->h64) {
        lv.c = make_coef<double>(lv.n, beta);
        launch_schur_diag<double>(h->st, lv.n, lv.c, lv.sinv, h->dom);
    }
    for (auto& lv : h->h32) {
        lv.c = make_coef<float>(lv.n, beta);
        const int k = (int)(&lv - h->h32.data());
        if (k <= h->small_top)   // the cooperative cycle's copy (the host structure stays in the handle)
            CK(cudaMemcpyAsync(h->dcoef + k, &lv.c, sizeof(OpCoef<float>), cudaMemcpyHostToDevice, h->st));
        // planar levels run only the register-tile step, which needs its coefficient structure
        if (lv.planar && !reg_tables_match(lv.c)) return STOKES_ERR_BAD_ARG;
        launch_schur_diag<float>(h->st, lv.n, make_coef<double>(lv.n, beta), lv.sinv, h->dom,
                                 lv.planar ? pl_vpitch(lv.n) : 0);
    }
    if (h->mixed()) {
        const OpCoef<double>& c = h->fin().c;
        const double* src = &c.A[0][0][0];
        float* hi = &h->chi.A[0][0][0];
        float* lo = &h->clo.A[0][0][0];
        const size_t cnt = sizeof(OpCoef<double>) / sizeof(double);
        for (size_t q = 0; q < cnt; ++q) {
            hi[q] = (float)src[q];
            lo[q] = (float)(src[q] - (double)hi[q]);
        }
    }
    CK(cudaGetLastError());
    double inv[27 * 27];
    if (!coarse_inverse(square_tables(), beta, inv)) return STOKES_ERR_BAD_ARG;
    CK(cudaMemcpyAsync(h->inv, inv, sizeof(inv), cudaMemcpyHostToDevice, h->st));
    if (h->clev > 0) {
        // the bordered system of the coarsest level, assembled on the host, inverted on the device
        std::vector<double> M((size_t)h->cnb * h->cnb);
        if (h->dom == kDomL) lshape_bordered_system(beta, M.data());   // the L's level 0 (square level 1)
        else bordered_system(square_tables(), 1 << (h->clev + 1), beta, M.data());
        CK(cudaMemcpyAsync(h->cinv, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
        CK(launch_dense_inverse(h->st, h->cinv, h->cnb, h->cperm, h->ccol, h->cstat));
        int st = 0;
        CK(cudaMemcpyAsync(&st, h->cstat, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        if (st != 0) return STOKES_ERR_BAD_ARG;
    }
    CK(cudaStreamSynchronize(h->st));
    if (h->step) {
        cudaGraphExecDestroy(h->step);
        h->step = nullptr;
    }
    if (h->loop) {
        cudaGraphExecDestroy(h->loop);
        h->loop = nullptr;
    }
    if (h->euler) {
        cudaGraphExecDestroy(h->euler);
        h->euler = nullptr;
    }
    return STOKES_OK;
}

stokes_status copy_in(stokes_handle* h, const double* u, const double* p, const double* f, const double* g) {
    Level<double>& F = h->fin();
    CK(cudaMemcpyAsync(F.u, u, 2 * F.n2 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(F.p, p, F.n1 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(F.f, f, 2 * F.n2 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(F.g, g, F.n1 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (h->dom == kDomL) {   // entries outside the L are ignored: they are zero from here on
        launch_mask_l(h->st, F.n, F.u, F.p);
        launch_mask_l(h->st, F.n, F.f, F.g);
        h->launches += 2;
    }
    return STOKES_OK;
}

stokes_status copy_out(stokes_handle* h, double* u, double* p) {
    Level<double>& F = h->fin();
    CK(cudaMemcpyAsync(u, F.u, 2 * F.n2 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(p, F.p, F.n1 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return STOKES_OK;
}

stokes_status read_scalar(stokes_handle* h, int idx, double* out) {
    CK(cudaMemcpyAsync(h->hscal + idx, h->scal + idx, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    *out = h->hscal[idx];
    return STOKES_OK;
}

}  // namespace

extern "C" {

void stokes_default_params(stokes_params* prm, int levels, double beta) {
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->levels = levels;
    prm->beta = beta;
    prm->nu_pre = 3;
    prm->nu_post = 3;
    prm->tau = 0.8;
    prm->sigma = 0.8;
    prm->smoother = STOKES_UZAWA;
    prm->gamma = 1;
    prm->precision = STOKES_FP64;
    prm->inner_cycles = 1;
    prm->coarse_level = 0;
    prm->domain = STOKES_UNIT_SQUARE;
}

const char* stokes_status_str(stokes_status s) {
    switch (s) {
        case STOKES_OK: return "ok";
        case STOKES_ERR_BAD_ARG: return "bad argument";
        case STOKES_ERR_OOM: return "out of device memory";
        case STOKES_ERR_CUDA: return "CUDA error";
        case STOKES_NOT_CONVERGED: return "not converged";
        case STOKES_DIVERGED: return "diverged";
        case STOKES_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

void stokes_destroy(stokes_handle* h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->step) cudaGraphExecDestroy(h->step);
    if (h->loop) cudaGraphExecDestroy(h->loop);
    if (h->euler) cudaGraphExecDestroy(h->euler);
    if (h->hhist) cudaFreeHost(h->hhist);
    for (auto e : h->ev) cudaEventDestroy(e);
    h->mem.put_all();   // level slabs, coarse inverses, partial sums, scalars, loop control, history
    if (h->hscal) cudaFreeHost(h->hscal);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
}

stokes_status stokes_setup(const stokes_params* prm, void* stream, stokes_handle** out) {
    ApiRange nvtx_range("stokes_setup");
    if (!prm || !out) return STOKES_ERR_BAD_ARG;
    *out = nullptr;
    const stokes_params& P = *prm;
    if (P.levels < 1 || P.levels > 13 || !(P.beta >= 0.0) || !std::isfinite(P.beta) || P.nu_pre < 0 ||
        P.nu_post < 0 || !(P.tau > 0.0) || !(P.sigma > 0.0) || (P.gamma != 1 && P.gamma != 2) ||
        (P.smoother != STOKES_UZAWA && P.smoother != STOKES_NORMAL_EQ) ||
        (P.precision != STOKES_FP64 && P.precision != STOKES_MIXED) ||
        (P.precision == STOKES_MIXED && P.inner_cycles < 1) || P.coarse_level < 0 ||
        P.coarse_level > kMaxCoarseLevel || P.coarse_level > P.levels - 1 ||
        (P.domain != STOKES_UNIT_SQUARE && P.domain != STOKES_L_SHAPE) || (P.tma_level != 0 && P.tma_level < 5) ||
        P.coop_level < -1 || P.coop_level > kSmallCycleTop)
        return STOKES_ERR_BAD_ARG;
    // the L-shaped domain: Uzawa cycles (float64, or float32 inside float64 refinement), coarsest
    // level 1 (the L's level 0)
    if (P.domain == STOKES_L_SHAPE && (P.smoother != STOKES_UZAWA || P.coarse_level != 1 || P.levels < 2))
        return STOKES_ERR_BAD_ARG;
    stokes_status s = ensure_weights();
    if (s != STOKES_OK) return s;
    if (prepare_uzawa_fused<float>() != cudaSuccess || prepare_uzawa_fused<double>() != cudaSuccess ||
        prepare_coarse_cycle() != cudaSuccess || prepare_uzawa_pair() != cudaSuccess ||
        prepare_uzawa_reg() != cudaSuccess || prepare_dense_solve(bordered_size(1 << (kMaxCoarseLevel + 1))) != cudaSuccess)
        return STOKES_ERR_CUDA;
    stokes_handle* h = new stokes_handle_t();
    h->prm = P;
    h->L = P.levels;
    if (stream) {
        h->st = (cudaStream_t)stream;
    } else {
        // a blocking stream: implicitly ordered with the legacy default stream, but capturable
        if (cudaStreamCreate(&h->st) != cudaSuccess) {
            delete h;
            return STOKES_ERR_CUDA;
        }
        h->own_stream = true;
    }
    auto bail = [&](stokes_status e) {
        stokes_destroy(h);
        return e;
    };
    init_mem(h->mem, h->st);
    h->dom = P.domain == STOKES_L_SHAPE ? kDomL : kDomSquare;
    const int kfin = P.levels - 1;
    if (P.precision == STOKES_FP64) {
        h->h64.resize(P.levels);
        for (int k = 0; k < P.levels; ++k)
            if ((s = alloc_level(h->h64[k], k, h->mem)) != STOKES_OK) return bail(s);
    } else {
        h->h64.resize(1);
        if ((s = alloc_level(h->h64[0], kfin, h->mem)) != STOKES_OK) return bail(s);
        h->h32.resize(P.levels);
        const int tlev = P.tma_level > 0 ? P.tma_level : kDefaultTmaLevel;
        const bool tma = P.smoother == STOKES_UZAWA && P.domain == STOKES_UNIT_SQUARE && uzawa_tma_available();
        for (int k = 0; k < P.levels; ++k)
            if ((s = alloc_level(h->h32[k], k, h->mem, tma && k >= tlev)) != STOKES_OK) return bail(s);
        h->has_planar = tma && tlev < P.levels;
        h->fuse_prolong = h->has_planar && fuse_prolong_enabled() && uzawa_tma_embed_available();
        // the cooperative small-level cycle: compact float32 levels up to coop_level, above the coarsest
        if (P.coop_level > 0 && P.smoother == STOKES_UZAWA && P.domain == STOKES_UNIT_SQUARE) {
            int top = P.coop_level;
            top = std::min(std::min(top, (int)kSmallCycleTop), std::min(P.levels - 1, tma ? tlev - 1 : (int)kSmallCycleTop));
            if (top > P.coarse_level) {
                h->small_top = top;
                if (h->mem.get(&h->dcoef, sizeof(OpCoef<float>) * (size_t)(top + 1)) != cudaSuccess ||
                    h->mem.get(&h->dbar, sizeof(unsigned)) != cudaSuccess) {
                    cudaGetLastError();
                    return bail(STOKES_ERR_OOM);
                }
            }
        }
    }
    h->mass = make_mass<double>(h->fin().n);
    h->npartial = 2 * cells_blocks(h->fin().n);   // two sets of per-block partial sums (refinement update)
    if (h->mem.get(&h->inv, 27 * 27 * sizeof(double)) != cudaSuccess ||
        h->mem.get(&h->partial, (size_t)h->npartial * sizeof(double)) != cudaSuccess ||
        h->mem.get(&h->scal, 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->hscal, 8 * sizeof(double)) != cudaSuccess ||
        h->mem.get(&h->dctl, 4 * sizeof(double)) != cudaSuccess || h->mem.get(&h->ictl, 4 * sizeof(int)) != cudaSuccess ||
        h->mem.get(&h->dhist, stokes_handle_t::kHistCap * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->hhist, stokes_handle_t::kHistCap * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bail(STOKES_ERR_OOM);
    }
    h->clev = P.coarse_level;
    if (h->clev > 0) {
        h->cnb = bordered_size(1 << (h->clev + 1));
        if (h->mem.get(&h->cinv, sizeof(double) * (size_t)h->cnb * h->cnb) != cudaSuccess ||
            h->mem.get(&h->cperm, sizeof(int) * (size_t)h->cnb) != cudaSuccess ||
            h->mem.get(&h->ccol, sizeof(double) * (size_t)h->cnb) != cudaSuccess ||
            h->mem.get(&h->cstat, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return bail(STOKES_ERR_OOM);
        }
    }
    if ((s = rebuild_beta(h)) != STOKES_OK) return bail(s);
    *out = h;
    return STOKES_OK;
}

static stokes_status autotune_levels(stokes_handle* h, cudaStream_t st);

stokes_status stokes_autotune(stokes_handle* h) {
    ApiRange nvtx_range("stokes_autotune");
    if (!h) return STOKES_ERR_BAD_ARG;
    stokes_status s = autotune_levels(h, h->st);
    if (s == STOKES_OK && h->step) {   // the captured cycle holds the old choices
        cudaGraphExecDestroy(h->step);
        h->step = nullptr;
    }
    if (s == STOKES_OK && h->loop) {
        cudaGraphExecDestroy(h->loop);
        h->loop = nullptr;
    }
    if (s == STOKES_OK && h->euler) {
        cudaGraphExecDestroy(h->euler);
        h->euler = nullptr;
    }
    return s;
}

stokes_status stokes_set_allocator(stokes_alloc_fn alloc, stokes_free_fn release, void* ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return STOKES_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_release = release;
    g_alloc_ctx = alloc ? ctx : nullptr;
    return STOKES_OK;
}

stokes_status stokes_set_beta(stokes_handle* h, double beta) {
    ApiRange nvtx_range("stokes_set_beta");
    if (!h || !(beta >= 0.0) || !std::isfinite(beta)) return STOKES_ERR_BAD_ARG;
    h->prm.beta = beta;
    return rebuild_beta(h);
}

stokes_status stokes_sizes(const stokes_handle* h, int* N, size_t* n_vel, size_t* n_p, size_t* ndof) {
    if (!h) return STOKES_ERR_BAD_ARG;
    const int n = 1 << h->L;
    if (N) *N = n;
    if (n_vel) *n_vel = 2 * (size_t)(2 * n + 1) * (2 * n + 1);
    if (n_p) *n_p = (size_t)(n + 1) * (n + 1);
    if (ndof) *ndof = 2 * (size_t)(2 * n - 1) * (2 * n - 1) + (size_t)(n + 1) * (n + 1);
    return STOKES_OK;
}

stokes_status stokes_cycle(stokes_handle* h, double* u, double* p, const double* f, const double* g) {
    ApiRange nvtx_range("stokes_cycle");
    if (!h || !u || !p || !f || !g) return STOKES_ERR_BAD_ARG;
    stokes_status s;
    if ((s = copy_in(h, u, p, f, g)) != STOKES_OK) return s;
    if (h->mixed()) {
        residual_norm_fin(h);   // float64 residual and the float32 right-hand side of the correction
        h->launches += 2;
    }
    if ((s = build_graph(h)) != STOKES_OK) return s;
    stokes_status s2 = launch_step(h);
    if (s2 != STOKES_OK) return s2;
    return take_launch_failure(h, copy_out(h, u, p));
}

stokes_status stokes_solve(stokes_handle* h, double* u, double* p, const double* f, const double* g,
                           double tol, int max_cycles, stokes_report* rep, double* history) {
    ApiRange nvtx_range("stokes_solve");
    if (!h || !u || !p || !f || !g || max_cycles < 0 || !(tol >= 0.0)) return STOKES_ERR_BAD_ARG;
    stokes_status s;
    if ((s = copy_in(h, u, p, f, g)) != STOKES_OK) return s;
    if ((s = build_graph(h)) != STOKES_OK) return s;
    Level<double>& F = h->fin();
    double nF2 = 0.0;
    launch_rhs_norm(h->st, F.n, F.f, F.g, h->partial);
    launch_reduce(h->st, h->partial, cells_blocks(F.n), h->scal + 2);
    h->launches += 2;
    if ((s = read_scalar(h, 2, &nF2)) != STOKES_OK) return s;
    const double nF = std::sqrt(nF2);
    residual_norm_fin(h);
    h->launches += 2;

    double r2 = 0.0;
    if ((s = read_scalar(h, 0, &r2)) != STOKES_OK) return s;
    double r0 = std::sqrt(r2), r = r0;
    if (history) history[0] = r0;
    int cycles = 0, grow_run = 0;
    double prev_r = r;
    stokes_status result = STOKES_OK;
    if (!h->timing) {
        // device-side loop: the host waits once per graph launch instead of once per cycle
        if ((s = build_loop(h)) != STOKES_OK) return s;
        for (;;) {
            if (r <= tol * nF) {
                if (!h->mixed()) break;
                residual_norm_fin(h);     // the updated residual of the refinement: confirm it
                h->launches += 2;
                if ((s = read_scalar(h, 0, &r2)) != STOKES_OK) return s;
                r = std::sqrt(r2);
                if (history) history[cycles] = r;
                if (r <= tol * nF) break;
            }
            if (!std::isfinite(r)) {
                result = STOKES_DIVERGED;
                break;
            }
            if (cycles >= max_cycles) {
                result = STOKES_NOT_CONVERGED;
                break;
            }
            // the device loop stops on the (updated) residual; MIXED then confirms with the true one
            double ctl[3] = {tol * tol, (double)(max_cycles - cycles), r * r};
            int ictl[2] = {0, 0};
            CK(cudaMemcpyAsync(h->dctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, h->st));
            CK(cudaMemcpyAsync(h->ictl, ictl, sizeof(ictl), cudaMemcpyHostToDevice, h->st));
            CK(cudaGraphLaunch(h->loop, h->st));
            CK(cudaMemcpyAsync(ictl, h->ictl, sizeof(ictl), cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            const int done = ictl[0];
            CK(cudaMemcpyAsync(h->hhist, h->dhist, sizeof(double) * std::min(done + 1, stokes_handle_t::kHistCap),
                               cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            h->launches += (unsigned long long)done * (h->loop_kernels);
            for (int c = 1; c <= done; ++c) {
                const double rc = c < stokes_handle_t::kHistCap ? std::sqrt(h->hhist[c]) : r;
                if (history) history[cycles + c] = rc;
            }
            cycles += done;
            r = done < stokes_handle_t::kHistCap ? std::sqrt(h->hhist[done]) : r;
            if (ictl[1] >= 8) {
                result = STOKES_DIVERGED;
                break;
            }
            if (done == 0) break;   // nothing ran (cannot happen with the default condition 1)
        }
    } else {
        for (;;) {
            if (r <= tol * nF) {
                if (!h->mixed()) break;
                // the refinement residual is updated, not recomputed: confirm with the true one
                residual_norm_fin(h);
                h->launches += 2;
                if ((s = read_scalar(h, 0, &r2)) != STOKES_OK) return s;
                r = std::sqrt(r2);
                if (history) history[cycles] = r;
                if (r <= tol * nF) break;
            }
            // diverged: NaN/Inf, or growth in each of the last 8 cycles (the first cycles from x = 0
            // may raise the Euclidean residual by orders of magnitude before it decays)
            grow_run = (cycles > 0 && r > prev_r) ? grow_run + 1 : 0;
            prev_r = r;
            if (!std::isfinite(r) || grow_run >= 8) {
                result = STOKES_DIVERGED;
                break;
            }
            if (cycles >= max_cycles) {
                result = STOKES_NOT_CONVERGED;
                break;
            }
            if ((s = launch_step(h)) != STOKES_OK) return s;
            if ((s = read_scalar(h, 0, &r2)) != STOKES_OK) return s;
            collect_timing(h);
            r = std::sqrt(r2);
            ++cycles;
            if (history) history[cycles] = r;
        }
    }
    if ((s = copy_out(h, u, p)) != STOKES_OK) return s;
    CK(cudaStreamSynchronize(h->st));
    if (rep) {
        rep->cycles = cycles;
        rep->rhs_norm = nF;
        rep->initial_residual = r0;
        rep->rel_residual = nF > 0 ? r / nF : r;
        rep->mean_rate = cycles > 0 && r0 > 0 ? std::pow(r / r0, 1.0 / cycles) : 0.0;
    }
    return take_launch_failure(h, result);
}

stokes_status stokes_residual(stokes_handle* h, const double* u, const double* p, const double* f,
                              const double* g, double* ru, double* rp) {
    if (!h || !u || !p || !f || !g || !ru || !rp) return STOKES_ERR_BAD_ARG;
    Level<double>& F = h->fin();
    launch_residual<double, double>(h->st, F.n, F.c, u, p, f, g, ru, rp, nullptr, nullptr, nullptr, h->dom);
    h->launches += 1;
    CK(cudaGetLastError());
    return STOKES_OK;
}

stokes_status stokes_residual_norm(stokes_handle* h, const double* u, const double* p, const double* f,
                                   const double* g, double* norm) {
    if (!h || !u || !p || !f || !g || !norm) return STOKES_ERR_BAD_ARG;
    Level<double>& F = h->fin();
    launch_residual<double, double>(h->st, F.n, F.c, u, p, f, g, F.tu, F.tp, h->partial, nullptr, nullptr, h->dom);
    launch_reduce(h->st, h->partial, cells_blocks(F.n), h->scal + 3);
    h->launches += 2;
    double v;
    stokes_status s = read_scalar(h, 3, &v);
    if (s != STOKES_OK) return s;
    *norm = std::sqrt(v);
    return STOKES_OK;
}

stokes_status stokes_smooth(stokes_handle* h, double* u, double* p, const double* f, const double* g, int nu) {
    if (!h || !u || !p || !f || !g || nu < 0) return STOKES_ERR_BAD_ARG;
    Level<double> lv = h->fin();   // coefficients, diagonals and temporaries of the finest level
    lv.u = u;
    lv.p = p;
    lv.f = const_cast<double*>(f);
    lv.g = const_cast<double*>(g);
    smooth_level<double>(h, lv, nu, false, false);
    h->launches += 3ull * nu;
    CK(cudaGetLastError());
    return STOKES_OK;
}

stokes_status stokes_smooth_f32(stokes_handle* h, float* u, float* p, const float* f, const float* g, int nu) {
    ApiRange nvtx_range("stokes_smooth_f32");
    if (!h || !u || !p || !f || !g || nu < 0 || !h->mixed()) return STOKES_ERR_BAD_ARG;
    Level<float> lv = h->h32.back();   // coefficients, diagonals and ping-pong partners of the finest level
    if (lv.planar) {
        // the caller's compact arrays into the level's own planar buffers, and the result back
        launch_to_planar(h->st, lv.n, u, p, lv.u, lv.p);
        launch_to_planar(h->st, lv.n, f, g, lv.f, lv.g);
        const bool sw = smooth_level<float>(h, lv, nu, false, false);
        launch_from_planar(h->st, lv.n, sw ? lv.tu : lv.u, sw ? lv.tp : lv.p, u, p);
        h->launches += (unsigned long long)nu + 3;
        CK(cudaGetLastError());
        return take_launch_failure(h);
    }
    lv.u = u;
    lv.p = p;
    lv.f = const_cast<float*>(f);
    lv.g = const_cast<float*>(g);
    const bool sw = smooth_level<float>(h, lv, nu, false, false);
    if (sw) {
        CK(cudaMemcpyAsync(u, lv.tu, 2 * lv.n2 * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(p, lv.tp, lv.n1 * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
    }
    h->launches += (unsigned long long)nu;
    CK(cudaGetLastError());
    return take_launch_failure(h);
}

stokes_status stokes_residual_restrict_f32(stokes_handle* h, const float* u, const float* p, const float* f,
                                           const float* g, float* fc, float* gc) {
    ApiRange nvtx_range("stokes_residual_restrict_f32");
    if (!h || !u || !p || !f || !g || !fc || !gc || !h->mixed() || h->L < 2) return STOKES_ERR_BAD_ARG;
    Level<float>& lv = h->h32.back();
    Level<float>& cl = h->h32[h->L - 2];
    if (lv.planar) {
        launch_to_planar(h->st, lv.n, u, p, lv.u, lv.p);
        launch_to_planar(h->st, lv.n, f, g, lv.f, lv.g);
        if (!launch_restrict_tma(h->st, lv.n, cl.planar, lv.c, lv.u, lv.p, lv.f, lv.g, cl.f, cl.g, cl.u, cl.p))
            return STOKES_ERR_CUDA;
        if (cl.planar) {
            launch_from_planar(h->st, cl.n, cl.f, cl.g, fc, gc);
        } else {
            CK(cudaMemcpyAsync(fc, cl.f, 2 * cl.n2 * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
            CK(cudaMemcpyAsync(gc, cl.g, cl.n1 * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
        }
        h->launches += 4;
    } else {
        launch_residual<float, float>(h->st, lv.n, lv.c, u, p, f, g, lv.tu, lv.tp, nullptr);
        launch_restrict<float>(h->st, cl.n, lv.tu, lv.tp, fc, gc);
        h->launches += 2;
    }
    CK(cudaGetLastError());
    return take_launch_failure(h);
}

stokes_status stokes_restrict(stokes_handle* h, const double* fu, const double* fp, double* fc, double* gc) {
    if (!h || !fu || !fp || !fc || !gc || h->L < 2) return STOKES_ERR_BAD_ARG;
    launch_restrict<double>(h->st, h->fin().n / 2, fu, fp, fc, gc, nullptr, nullptr, h->dom);
    h->launches += 1;
    CK(cudaGetLastError());
    return STOKES_OK;
}

stokes_status stokes_prolong_add(stokes_handle* h, const double* uc, const double* pc, double* uf, double* pf) {
    if (!h || !uc || !pc || !uf || !pf || h->L < 2) return STOKES_ERR_BAD_ARG;
    launch_prolong_add<double>(h->st, h->fin().n / 2, uc, pc, uf, pf, h->dom);
    h->launches += 1;
    CK(cudaGetLastError());
    return STOKES_OK;
}

stokes_status stokes_load_vectors(stokes_handle* h, const double* f_nodal, const double* g_nodal, int project_g,
                                  double* f, double* g) {
    if (!h || !f_nodal || !g_nodal || !f || !g || h->dom != kDomSquare) return STOKES_ERR_BAD_ARG;
    launch_load<double>(h->st, h->fin().n, h->mass, f_nodal, g_nodal, f, g, project_g, h->partial, h->scal + 4);
    h->launches += project_g ? 3 : 1;
    CK(cudaGetLastError());
    return STOKES_OK;
}

stokes_status stokes_stencil_class(int levels, int i, int j, int* cls) {
    if (levels < 1 || levels > 13 || !cls) return STOKES_ERR_BAD_ARG;
    const int n = 1 << levels;
    if (i < 0 || j < 0 || i > n || j > n) return STOKES_ERR_BAD_ARG;
    *cls = stencil_class(i, j, n);
    return STOKES_OK;
}

stokes_status stokes_stencil_rows(int levels, double beta, int cls, double* ma, double* mbtx, double* mbty,
                                  double* mbx, double* mby, double* midg) {
    if (levels < 1 || levels > 13 || !(beta >= 0.0) || !std::isfinite(beta) || cls < 0 || cls >= kStencilClasses ||
        !ma || !mbtx || !mbty || !mbx || !mby || !midg)
        return STOKES_ERR_BAD_ARG;
    const OpCoef<double> c = make_coef<double>(1 << levels, beta);
    std::memcpy(ma, c.MA[cls], sizeof(c.MA[cls]));
    std::memcpy(mbtx, c.MBTx[cls], sizeof(c.MBTx[cls]));
    std::memcpy(mbty, c.MBTy[cls], sizeof(c.MBTy[cls]));
    std::memcpy(mbx, c.MBx[cls], sizeof(c.MBx[cls]));
    std::memcpy(mby, c.MBy[cls], sizeof(c.MBy[cls]));
    std::memcpy(midg, c.MIdg[cls], sizeof(c.MIdg[cls]));
    return STOKES_OK;
}

stokes_status stokes_step_tables_match(int levels, double beta) {
    if (levels < 1 || levels > 13 || !(beta >= 0.0) || !std::isfinite(beta)) return STOKES_ERR_BAD_ARG;
    return reg_tables_match(make_coef<float>(1 << levels, beta)) ? STOKES_OK : STOKES_ERR_BAD_ARG;
}

stokes_status stokes_transfer_weights(double* w) {
    if (!w) return STOKES_ERR_BAD_ARG;
    const TransferWeights W = transfer_weights();
    std::memcpy(w, &W.P2[0][0][0][0], sizeof(W.P2));
    return STOKES_OK;
}

stokes_status stokes_embed_weights(double* w) {
    if (!w) return STOKES_ERR_BAD_ARG;
    embed_weights_table(w);
    return STOKES_OK;
}

stokes_status stokes_coarse_inverse(double beta, double* inv) {
    if (!inv || !(beta >= 0.0) || !std::isfinite(beta)) return STOKES_ERR_BAD_ARG;
    return coarse_inverse(square_tables(), beta, inv) ? STOKES_OK : STOKES_ERR_BAD_ARG;
}

stokes_status stokes_euler_rhs(stokes_handle* h, const double* u_prev, const double* f_nodal, const double* g_nodal,
                               double* f, double* g) {
    if (!h || !u_prev || !f_nodal || !g_nodal || !f || !g || h->dom != kDomSquare) return STOKES_ERR_BAD_ARG;
    const int n = h->fin().n;
    const size_t nvel = 2 * (size_t)(2 * n + 1) * (2 * n + 1);
    if (!h->euler_w) CK(h->mem.get(&h->euler_w, nvel * sizeof(double)));
    CK(launch_euler_nodal(h->st, nvel, h->prm.beta, f_nodal, u_prev, h->euler_w));
    launch_load<double>(h->st, n, h->mass, h->euler_w, g_nodal, f, g, 1, h->partial, h->scal + 4);
    h->launches += 4;
    CK(cudaGetLastError());
    return STOKES_OK;
}

stokes_status stokes_make_consistent(stokes_handle* h, double* g) {
    if (!h || !g || h->dom != kDomSquare) return STOKES_ERR_BAD_ARG;
    launch_make_consistent(h->st, h->fin().n, g, h->partial, h->scal + 6);
    h->launches += 3;
    CK(cudaGetLastError());
    return STOKES_OK;
}

stokes_status stokes_mass_dot(stokes_handle* h, const double* a, const double* b, double* dot) {
    if (!h || !a || !b || !dot || h->dom != kDomSquare) return STOKES_ERR_BAD_ARG;
    const int n = h->fin().n;
    launch_mass_dot(h->st, n, h->mass, a, b, h->partial);
    launch_reduce(h->st, h->partial, cells_blocks(n), h->scal + 5);
    h->launches += 2;
    return read_scalar(h, 5, dot);
}

stokes_status stokes_set_timing(stokes_handle* h, int enable) {
    if (!h) return STOKES_ERR_BAD_ARG;
    const bool on = enable != 0;
    if (on && h->ev.empty()) {
        const int pairs = (h->prm.nu_pre + h->prm.nu_post) * (h->mixed() ? h->prm.inner_cycles : 1) + 1;
        h->ev.resize(2 * pairs);
        h->ev_kind.assign(pairs, kEvSmooth);
        for (auto& e : h->ev) CK(cudaEventCreate(&e));
    }
    if (on != h->timing && h->step) {
        cudaGraphExecDestroy(h->step);
        h->step = nullptr;
    }
    h->timing = on;
    h->t_smooth = h->t_resid = h->t_fused = 0.0;
    h->n_smooth = h->n_resid = h->n_fused = 0;
    return STOKES_OK;
}

stokes_status stokes_get_timing(const stokes_handle* h, double* smooth_ms, long long* smooth_count,
                                double* resid_ms, long long* resid_count) {
    if (!h) return STOKES_ERR_BAD_ARG;
    if (smooth_ms) *smooth_ms = h->t_smooth;
    if (smooth_count) *smooth_count = h->n_smooth;
    if (resid_ms) *resid_ms = h->t_resid;
    if (resid_count) *resid_count = h->n_resid;
    return STOKES_OK;
}

stokes_status stokes_get_timing_fused(const stokes_handle* h, double* ms, long long* count) {
    if (!h) return STOKES_ERR_BAD_ARG;
    if (ms) *ms = h->t_fused;
    if (count) *count = h->n_fused;
    return STOKES_OK;
}

unsigned long long stokes_kernel_launches(const stokes_handle* h) { return h ? h->launches : 0ull; }

// ----------------------------------------------------------------------------------- batches

// Times the float32 Uzawa step variants on each not-yet-tuned level of h's float32 hierarchy
// (process-wide choice per level size) and leaves the buffers zero as a fresh handle has them.
static stokes_status autotune_levels(stokes_handle* h, cudaStream_t st) {
    // the L's float32 levels run the per-phase step only: nothing to choose
    if (!h->mixed() || h->prm.smoother != STOKES_UZAWA || h->dom != kDomSquare) return STOKES_OK;
    for (int l = 1; l < (int)h->h32.size(); ++l) {
        Level<float>& lv = h->h32[l];
        if (lv.planar ? tma_tuned(lv.n) : uzawa_tuned(lv.n)) continue;
        cudaError_t e = lv.planar ? autotune_uzawa_tma(st, lv.n, lv.c, (float)h->prm.tau, (float)h->prm.sigma, lv.u, lv.p,
                                                       lv.f, lv.g, lv.sinv, lv.tu, lv.tp)
                                  : autotune_uzawa_fused(st, lv.n, lv.c, (float)h->prm.tau, (float)h->prm.sigma, lv.u,
                                                         lv.p, lv.f, lv.g, lv.sinv, lv.tu, lv.tp, nullptr, nullptr);
        if (e != cudaSuccess) return fail(e);
        cudaMemsetAsync(lv.u, 0, 2 * lv.n2 * sizeof(float), st);
        cudaMemsetAsync(lv.p, 0, lv.n1 * sizeof(float), st);
        cudaMemsetAsync(lv.tu, 0, 2 * lv.n2 * sizeof(float), st);
        cudaMemsetAsync(lv.tp, 0, lv.n1 * sizeof(float), st);
    }
    CK(cudaStreamSynchronize(st));
    return STOKES_OK;
}

int stokes_step_variant(int levels) { return levels >= 2 && levels <= 31 ? uzawa_choice(1 << levels) : -1; }

stokes_status stokes_set_step_variant(int levels, int variant) {
    if (levels < 2 || levels > 31 || !set_uzawa_choice(1 << levels, variant)) return STOKES_ERR_BAD_ARG;
    return STOKES_OK;
}

int stokes_planar_step_variant(int levels) { return levels >= 2 && levels <= 31 ? tma_choice(1 << levels) : -1; }

stokes_status stokes_set_planar_step_variant(int levels, int variant) {
    if (levels < 2 || levels > 31 || !set_tma_choice(1 << levels, variant)) return STOKES_ERR_BAD_ARG;
    return STOKES_OK;
}

struct stokes_batch_t {
    int count = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<stokes_handle*> inst;
    std::vector<int> body_kernels;      // kernels per loop iteration of each instance
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;       // pointers, tol and max_cycles the graph was built for
    double tol = -1.0;
    int max_cycles = -1;
    int* d_count = nullptr;             // device: refinement steps per instance
    double* d_res = nullptr;            // device: per instance (true ||r||^2, ||F||^2, steps)
    double* h_res = nullptr;            // pinned mirror
    unsigned long long launches = 0;
    DevMem mem;
};

void stokes_batch_destroy(stokes_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto h : b->inst) stokes_destroy(h);
    b->mem.put_all();
    if (b->h_res) cudaFreeHost(b->h_res);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

stokes_status stokes_batch_setup(int count, const int* levels, const double* betas, const stokes_params* base,
                                 void* stream, int autotune, stokes_batch** out) {
    ApiRange nvtx_range("stokes_batch_setup");
    if (count < 1 || !levels || !betas || !base || !out) return STOKES_ERR_BAD_ARG;
    *out = nullptr;
    stokes_batch* b = new stokes_batch_t();
    b->count = count;
    if (stream) {
        b->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreate(&b->st) != cudaSuccess) {
            delete b;
            return STOKES_ERR_CUDA;
        }
        b->own_stream = true;
    }
    stokes_status s;
    for (int i = 0; i < count; ++i) {
        stokes_params prm = *base;
        prm.levels = levels[i];
        prm.beta = betas[i];
        stokes_handle* h = nullptr;
        if ((s = stokes_setup(&prm, b->st, &h)) != STOKES_OK) {
            stokes_batch_destroy(b);
            return s;
        }
        b->inst.push_back(h);
    }
    init_mem(b->mem, b->st);
    if (b->mem.get(&b->d_count, sizeof(int) * count) != cudaSuccess ||
        b->mem.get(&b->d_res, sizeof(double) * 3 * count) != cudaSuccess ||
        cudaMallocHost(&b->h_res, sizeof(double) * 3 * count) != cudaSuccess) {
        cudaGetLastError();
        stokes_batch_destroy(b);
        return STOKES_ERR_OOM;
    }
    if (autotune) {
        for (auto h : b->inst)
            if ((s = autotune_levels(h, b->st)) != STOKES_OK) {
                stokes_batch_destroy(b);
                return s;
            }
    }
    *out = b;
    return STOKES_OK;
}

static stokes_status batch_build(stokes_batch* b, double* const* u, double* const* p, const double* const* f,
                                 const double* const* g, double tol, int max_cycles) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaStream_t st = b->st;
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0));
    b->body_kernels.assign(b->count, 0);
    auto count_kernels = [](cudaGraph_t gr) {
        size_t nn = 0;
        cudaGraphGetNodes(gr, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(gr, nodes.data(), &nn);
        int k = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
        }
        return k;
    };
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
        stokes_handle* h = b->inst[i];
        Level<double>& F = h->fin();
        const bool mixed = h->mixed();
        // prologue: inputs in, ||F||, true residual, step counter
        cudaGraph_t gp = nullptr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        copy_in(h, u[i], p[i], f[i], g[i]);
        launch_rhs_norm(st, F.n, F.f, F.g, h->partial);
        launch_reduce(st, h->partial, cells_blocks(F.n), h->scal + 2);
        residual_norm_fin(h);
        cudaMemsetAsync(b->d_count + i, 0, sizeof(int), st);
        if ((e = cudaStreamEndCapture(st, &gp)) != cudaSuccess) break;
        cudaGraphNode_t np, nc, ne;
        e = cudaGraphAddChildGraphNode(&np, top, nullptr, 0, gp);
        cudaGraphDestroy(gp);
        if (e != cudaSuccess) break;
        // loop: WHILE the step's residual is above the tolerance (MIXED: the updated residual; the
        // epilogue computes the true one, and the rare instance that misses continues on the host)
        cudaGraphConditionalHandle hnd;
        if ((e = cudaGraphConditionalHandleCreate(&hnd, top, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hnd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if ((e = cudaGraphAddNode(&nc, top, &np, nullptr, 1, &cp)) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            break;
        record_step(h);
        launch_batch_check(st, hnd, h->scal, tol * tol, max_cycles, b->d_count + i);
        if ((e = cudaStreamEndCapture(st, &body)) != cudaSuccess) break;
        b->body_kernels[i] = count_kernels(body);
        // epilogue: true residual, results out
        cudaGraph_t ge = nullptr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        residual_norm_fin(h);
        launch_batch_store(st, h->scal, b->d_count + i, b->d_res + 3 * i);
        copy_out(h, u[i], p[i]);
        if ((e = cudaStreamEndCapture(st, &ge)) != cudaSuccess) break;
        e = cudaGraphAddChildGraphNode(&ne, top, &nc, 1, ge);
        cudaGraphDestroy(ge);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, top, 0);
    cudaGraphDestroy(top);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return fail(e);
    }
    return STOKES_OK;
}

stokes_status stokes_batch_solve(stokes_batch* b, double* const* u, double* const* p, const double* const* f,
                                 const double* const* g, double tol, int max_cycles, int* cycles,
                                 double* rel_residual) {
    ApiRange nvtx_range("stokes_batch_solve");
    if (!b || !u || !p || !f || !g || !(tol > 0.0) || max_cycles < 1) return STOKES_ERR_BAD_ARG;
    std::vector<const void*> key;
    for (int i = 0; i < b->count; ++i) {
        if (!u[i] || !p[i] || !f[i] || !g[i]) return STOKES_ERR_BAD_ARG;
        key.insert(key.end(), {u[i], p[i], f[i], g[i]});
    }
    stokes_status s;
    if (!b->exec || key != b->key || tol != b->tol || max_cycles != b->max_cycles) {
        if ((s = batch_build(b, u, p, f, g, tol, max_cycles)) != STOKES_OK) return s;
        b->key = key;
        b->tol = tol;
        b->max_cycles = max_cycles;
    }
    CK(cudaGraphLaunch(b->exec, b->st));
    CK(cudaMemcpyAsync(b->h_res, b->d_res, sizeof(double) * 3 * b->count, cudaMemcpyDeviceToHost, b->st));
    CK(cudaStreamSynchronize(b->st));
    stokes_status result = STOKES_OK;
    for (int i = 0; i < b->count; ++i) {
        stokes_handle* h = b->inst[i];
        const int steps = (int)b->h_res[3 * i + 2];
        const double nF = std::sqrt(b->h_res[3 * i + 1]);
        double r = std::sqrt(b->h_res[3 * i]);
        b->launches += 4 + 3 + (unsigned long long)steps * (b->body_kernels[i] + 1);
        int total = steps;
        if (!(r <= tol * nF)) {
            // rare: the true residual misses the tolerance; continue this instance on its own
            stokes_report rep{};
            const unsigned long long before = h->launches;
            stokes_status si = stokes_solve(h, u[i], p[i], f[i], g[i], tol, max_cycles > steps ? max_cycles - steps : 1,
                                            &rep, nullptr);
            b->launches += h->launches - before;
            total += rep.cycles;
            r = rep.rel_residual * nF;
            if (si != STOKES_OK && result == STOKES_OK) result = si;
        }
        if (cycles) cycles[i] = total;
        if (rel_residual) rel_residual[i] = nF > 0 ? r / nF : r;
    }
    for (int i = 0; i < b->count; ++i) result = take_launch_failure(b->inst[i], result);
    return result;
}

unsigned long long stokes_batch_kernel_launches(const stokes_batch* b) { return b ? b->launches : 0ull; }

// ----------------------------------------------------------------------------------- time stepping

static int graph_kernels(cudaGraph_t gr) {
    size_t nn = 0;
    cudaGraphGetNodes(gr, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(gr, nodes.data(), &nn);
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Appends to `top`, after *dep (null: no dependency), the implicit Euler steps of handle h (Sec. 1:
// the step of length dt is the generalized Stokes system with beta = 1/dt, the handle's beta): (u, p)
// is copied into the handle's finest arrays; per step n the right-hand side is formed from the nodal
// data f_nodal[n] + beta u and g_nodal[n] (load vectors, g shifted to zero mean), ||F||^2 and the
// true residual are computed, a conditional WHILE node runs cycles (body: one cycle, or one
// refinement step followed by the true float64 residual; then the device-side test of the relative
// residual against tol and of max_cycles), and the step's true ||r||^2, ||F||^2 and cycle count go to
// res[3 n .. 3 n + 2]; finally (u, p) is written back.  *kernels counts the kernels outside the loop
// bodies, *body those of one loop iteration.
static cudaError_t add_euler_chain(cudaGraph_t top, cudaGraphNode_t* dep, stokes_handle* h, double* u, double* p,
                                   const double* const* f_nodal, const double* const* g_nodal, int steps,
                                   double tol, int max_cycles, int* count, double* res, int* kernels, int* body) {
    cudaStream_t st = h->st;
    Level<double>& F = h->fin();
    const size_t nvel = 2 * F.n2;
    const bool timing = h->timing;
    h->timing = false;
    cudaError_t e = cudaSuccess;
    auto child = [&](auto&& record) -> cudaError_t {
        cudaGraph_t g = nullptr;
        cudaError_t r = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (r != cudaSuccess) return r;
        record();
        if ((r = cudaStreamEndCapture(st, &g)) != cudaSuccess) return r;
        *kernels += graph_kernels(g);
        cudaGraphNode_t nd;
        r = cudaGraphAddChildGraphNode(&nd, top, *dep ? dep : nullptr, *dep ? 1 : 0, g);
        cudaGraphDestroy(g);
        if (r == cudaSuccess) *dep = nd;
        return r;
    };
    e = child([&] {
        cudaMemcpyAsync(F.u, u, nvel * sizeof(double), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(F.p, p, F.n1 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    });
    for (int n = 0; n < steps && e == cudaSuccess; ++n) {
        e = child([&] {
            launch_euler_nodal(st, nvel, h->prm.beta, f_nodal[n], F.u, h->euler_w);
            launch_load<double>(st, F.n, h->mass, h->euler_w, g_nodal[n], F.f, F.g, 1, h->partial, h->scal + 4);
            launch_rhs_norm(st, F.n, F.f, F.g, h->partial);
            launch_reduce(st, h->partial, cells_blocks(F.n), h->scal + 2);
            residual_norm_fin(h);
            cudaMemsetAsync(count + n, 0, sizeof(int), st);
        });
        if (e != cudaSuccess) break;
        cudaGraphConditionalHandle hnd;
        if ((e = cudaGraphConditionalHandleCreate(&hnd, top, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hnd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t nc;
        if ((e = cudaGraphAddNode(&nc, top, dep, nullptr, 1, &cp)) != cudaSuccess) break;
        cudaGraph_t bg = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(st, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            break;
        record_step(h);
        if (h->mixed()) residual_norm_fin(h);   // the test uses the true residual, not the updated one
        launch_batch_check(st, hnd, h->scal, tol * tol, max_cycles, count + n);
        if ((e = cudaStreamEndCapture(st, &bg)) != cudaSuccess) break;
        *body = graph_kernels(bg);
        *dep = nc;
        e = child([&] { launch_batch_store(st, h->scal, count + n, res + 3 * n); });
    }
    if (e == cudaSuccess)
        e = child([&] {
            cudaMemcpyAsync(u, F.u, nvel * sizeof(double), cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(p, F.p, F.n1 * sizeof(double), cudaMemcpyDeviceToDevice, st);
        });
    h->timing = timing;
    return e;
}

// reads back the per-step results of an Euler graph; OK, or NOT_CONVERGED if a step missed tol
static stokes_status euler_results(const std::vector<double>& res, int steps, double tol, int* cycles,
                                   double* rel_residual, unsigned long long* total_cycles) {
    stokes_status out = STOKES_OK;
    for (int n = 0; n < steps; ++n) {
        const double r = std::sqrt(res[3 * n]), nF = std::sqrt(res[3 * n + 1]);
        const int c = (int)res[3 * n + 2];
        *total_cycles += (unsigned long long)c;
        if (cycles) cycles[n] = c;
        const double rel = nF > 0 ? r / nF : r;
        if (rel_residual) rel_residual[n] = rel;
        if (!(rel <= tol)) out = STOKES_NOT_CONVERGED;
    }
    return out;
}

stokes_status stokes_euler_run(stokes_handle* h, double* u, double* p, const double* const* f_nodal,
                               const double* const* g_nodal, int steps, double tol, int max_cycles, int* cycles,
                               double* rel_residual) {
    ApiRange nvtx_range("stokes_euler_run");
    if (!h || !u || !p || !f_nodal || !g_nodal || steps < 1 || !(tol > 0.0) || max_cycles < 1) return STOKES_ERR_BAD_ARG;
    std::vector<const void*> key = {u, p};
    for (int n = 0; n < steps; ++n) {
        if (!f_nodal[n] || !g_nodal[n]) return STOKES_ERR_BAD_ARG;
        key.push_back(f_nodal[n]);
        key.push_back(g_nodal[n]);
    }
    Level<double>& F = h->fin();
    if (!h->euler_w) CK(h->mem.get(&h->euler_w, 2 * F.n2 * sizeof(double)));
    if (!h->euler || key != h->euler_key || tol != h->euler_tol || max_cycles != h->euler_max) {
        if (h->euler) {
            cudaGraphExecDestroy(h->euler);
            h->euler = nullptr;
        }
        CK(cudaStreamSynchronize(h->st));
        h->mem.put(h->d_ecount);
        h->mem.put(h->d_eres);
        h->d_ecount = nullptr;
        h->d_eres = nullptr;
        CK(h->mem.get(&h->d_ecount, sizeof(int) * (size_t)steps));
        CK(h->mem.get(&h->d_eres, sizeof(double) * 3 * (size_t)steps));
        cudaGraph_t top = nullptr;
        CK(cudaGraphCreate(&top, 0));
        cudaGraphNode_t dep = nullptr;
        h->euler_kernels = h->euler_body = 0;
        cudaError_t e = add_euler_chain(top, &dep, h, u, p, f_nodal, g_nodal, steps, tol, max_cycles, h->d_ecount,
                                        h->d_eres, &h->euler_kernels, &h->euler_body);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->euler, top, 0);
        cudaGraphDestroy(top);
        if (e != cudaSuccess) {
            h->euler = nullptr;
            return fail(e);
        }
        h->euler_key = key;
        h->euler_tol = tol;
        h->euler_max = max_cycles;
    }
    CK(cudaGraphLaunch(h->euler, h->st));
    std::vector<double> res(3 * (size_t)steps);
    CK(cudaMemcpyAsync(res.data(), h->d_eres, res.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    unsigned long long total = 0;
    const stokes_status out = euler_results(res, steps, tol, cycles, rel_residual, &total);
    h->launches += (unsigned long long)h->euler_kernels + total * (unsigned long long)h->euler_body;
    return take_launch_failure(h, out);
}

stokes_status stokes_batch_euler_run(stokes_batch* b, double* const* u, double* const* p,
                                     const double* const* f_nodal, const double* const* g_nodal, int steps,
                                     double tol, int max_cycles, int* cycles, double* rel_residual) {
    ApiRange nvtx_range("stokes_batch_euler_run");
    if (!b || !u || !p || !f_nodal || !g_nodal || steps < 1 || !(tol > 0.0) || max_cycles < 1)
        return STOKES_ERR_BAD_ARG;
    const int count = b->count;
    for (int i = 0; i < count; ++i) {
        if (!u[i] || !p[i]) return STOKES_ERR_BAD_ARG;
        for (int n = 0; n < steps; ++n)
            if (!f_nodal[(size_t)i * steps + n] || !g_nodal[(size_t)i * steps + n]) return STOKES_ERR_BAD_ARG;
    }
    // one graph per call: every instance's chain of steps is an independent branch
    std::vector<int*> dcount(count, nullptr);
    std::vector<double*> dres(count, nullptr);
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0));
    cudaError_t e = cudaSuccess;
    std::vector<int> kern(count, 0), body(count, 0);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        stokes_handle* h = b->inst[i];
        Level<double>& F = h->fin();
        if (!h->euler_w && (e = h->mem.get(&h->euler_w, 2 * F.n2 * sizeof(double))) != cudaSuccess) break;
        if ((e = b->mem.get(&dcount[i], sizeof(int) * (size_t)steps)) != cudaSuccess) break;
        if ((e = b->mem.get(&dres[i], sizeof(double) * 3 * (size_t)steps)) != cudaSuccess) break;
        // the instance's stream is the batch's stream: the branches are captured one after another
        cudaGraphNode_t dep = nullptr;
        e = add_euler_chain(top, &dep, h, u[i], p[i], f_nodal + (size_t)i * steps, g_nodal + (size_t)i * steps, steps,
                            tol, max_cycles, dcount[i], dres[i], &kern[i], &body[i]);
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, top, 0);
    cudaGraphDestroy(top);
    stokes_status out = STOKES_OK;
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->st);
    std::vector<double> res(3 * (size_t)steps);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        if ((e = cudaMemcpyAsync(res.data(), dres[i], res.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(b->st)) != cudaSuccess)
            break;
        unsigned long long total = 0;
        const stokes_status si = euler_results(res, steps, tol, cycles ? cycles + (size_t)i * steps : nullptr,
                                               rel_residual ? rel_residual + (size_t)i * steps : nullptr, &total);
        if (si != STOKES_OK) out = si;
        b->launches += (unsigned long long)kern[i] + total * (unsigned long long)body[i];
    }
    if (exec) {
        cudaStreamSynchronize(b->st);
        cudaGraphExecDestroy(exec);
    }
    for (int i = 0; i < count; ++i) {
        b->mem.put(dcount[i]);
        b->mem.put(dres[i]);
    }
    if (e != cudaSuccess) return fail(e);
    for (int i = 0; i < count; ++i) out = take_launch_failure(b->inst[i], out);
    return out;
}

}  // extern "C"
