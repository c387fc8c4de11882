"""Python front end of the CUDA solver: torch tensors in, torch tensors out.

Every step runs in the CUDA library (include/stokes_mg.h); this module only checks shapes and
passes device pointers and the current stream.

Layouts (float64, CUDA, contiguous):  u (2, 2N+1, 2N+1), p (N+1, N+1), with N = 2^levels.
"""
import ctypes
import math

import torch

from . import _binding as B

_SMOOTHERS = {"uzawa": B.UZAWA, "normal": B.NORMAL_EQ}
_PREC = {"fp64": B.FP64, "mixed": B.MIXED}
_DOMAINS = {"square": B.UNIT_SQUARE, "lshape": B.L_SHAPE}


class Report:
    def __init__(self, r: B.Report, history, status):
        self.cycles = r.cycles
        self.rel_residual = r.rel_residual
        self.mean_rate = r.mean_rate
        self.initial_residual = r.initial_residual
        self.rhs_norm = r.rhs_norm
        self.history = history
        self.status = status

    @property
    def converged(self):
        return self.status == B.OK

    def __repr__(self):
        return "Report(cycles=%d, rel_residual=%.3e, mean_rate=%.4f)" % (self.cycles, self.rel_residual, self.mean_rate)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """Coupled multigrid solver for [A + beta M, B^T; B, 0] on level k = levels - 1."""

    def __init__(self, levels: int, beta: float, *, nu_pre=3, nu_post=3, tau=None, sigma=0.8,
                 smoother="uzawa", gamma=1, precision="fp64", inner_cycles=1, coarse_level=0, domain="square",
                 tma_level=0, coop_level=0, stream=None, device=None):
        self._lib = B.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        prm = B.Params()
        self._lib.stokes_default_params(ctypes.byref(prm), levels, float(beta))
        prm.nu_pre, prm.nu_post = nu_pre, nu_post
        prm.smoother = _SMOOTHERS[smoother]
        prm.tau = (0.8 if smoother == "uzawa" else 0.35) if tau is None else tau
        prm.sigma = sigma
        prm.gamma = gamma
        prm.precision = _PREC[precision]
        prm.inner_cycles = inner_cycles
        prm.coarse_level = coarse_level
        prm.domain = _DOMAINS[domain]
        prm.tma_level = tma_level
        prm.coop_level = coop_level
        self.params = prm
        self.levels = levels
        self.beta = float(beta)
        self.N = 2 ** levels
        self.precision = precision
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream() if stream is None else stream
            self._stream = s
            h = ctypes.c_void_p()
            B.check(self._lib.stokes_setup(ctypes.byref(prm), ctypes.c_void_p(s.cuda_stream), ctypes.byref(h)),
                    "stokes_setup")
        self._h = h

    # ------------------------------------------------------------------ helpers
    @property
    def shape_u(self):
        return (2, 2 * self.N + 1, 2 * self.N + 1)

    @property
    def shape_p(self):
        return (self.N + 1, self.N + 1)

    @property
    def ndof(self):
        return 2 * (2 * self.N - 1) ** 2 + (self.N + 1) ** 2

    def _chk(self, t, shape, name):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.device != self.device \
                or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError("%s must be a contiguous float64 tensor of shape %s on %s" % (name, shape, self.device))
        return _ptr(t)

    def zeros_u(self):
        return torch.zeros(self.shape_u, dtype=torch.float64, device=self.device)

    def zeros_p(self):
        return torch.zeros(self.shape_p, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stokes_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ API
    def set_beta(self, beta):
        B.check(self._lib.stokes_set_beta(self._h, float(beta)), "stokes_set_beta")
        self.beta = float(beta)

    def load_vectors(self, f_nodal, g_nodal, project_g=True, out=None):
        """Load vectors (f, g) of nodal data; out = (f, g) writes into given float64 tensors."""
        if out is None:
            f, g = self.zeros_u(), self.zeros_p()
        else:
            f, g = out
            self._chk(f, self.shape_u, "f")
            self._chk(g, self.shape_p, "g")
        B.check(self._lib.stokes_load_vectors(self._h, self._chk(f_nodal, self.shape_u, "f_nodal"),
                                              self._chk(g_nodal, self.shape_p, "g_nodal"), int(project_g),
                                              _ptr(f), _ptr(g)), "stokes_load_vectors")
        return f, g

    def solve(self, f, g, tol=1e-10, max_cycles=100, u=None, p=None, raise_on_fail=False):
        u = self.zeros_u() if u is None else u
        p = self.zeros_p() if p is None else p
        rep = B.Report()
        hist = (ctypes.c_double * (max_cycles + 1))()
        st = self._lib.stokes_solve(self._h, self._chk(u, self.shape_u, "u"), self._chk(p, self.shape_p, "p"),
                                    self._chk(f, self.shape_u, "f"), self._chk(g, self.shape_p, "g"),
                                    float(tol), int(max_cycles), ctypes.byref(rep), hist)
        if st not in (B.OK, B.NOT_CONVERGED, B.DIVERGED) or (raise_on_fail and st != B.OK):
            B.check(st, "stokes_solve")
        return u, p, Report(rep, [hist[i] for i in range(rep.cycles + 1)], st)

    def cycle(self, u, p, f, g):
        B.check(self._lib.stokes_cycle(self._h, self._chk(u, self.shape_u, "u"), self._chk(p, self.shape_p, "p"),
                                       self._chk(f, self.shape_u, "f"), self._chk(g, self.shape_p, "g")),
                "stokes_cycle")
        return u, p

    def residual(self, u, p, f, g):
        ru, rp = self.zeros_u(), self.zeros_p()
        B.check(self._lib.stokes_residual(self._h, self._chk(u, self.shape_u, "u"), self._chk(p, self.shape_p, "p"),
                                          self._chk(f, self.shape_u, "f"), self._chk(g, self.shape_p, "g"),
                                          _ptr(ru), _ptr(rp)), "stokes_residual")
        return ru, rp

    def residual_norm(self, u, p, f, g):
        out = ctypes.c_double()
        B.check(self._lib.stokes_residual_norm(self._h, self._chk(u, self.shape_u, "u"),
                                               self._chk(p, self.shape_p, "p"), self._chk(f, self.shape_u, "f"),
                                               self._chk(g, self.shape_p, "g"), ctypes.byref(out)),
                "stokes_residual_norm")
        return out.value

    def smooth(self, u, p, f, g, nu=1):
        B.check(self._lib.stokes_smooth(self._h, self._chk(u, self.shape_u, "u"), self._chk(p, self.shape_p, "p"),
                                        self._chk(f, self.shape_u, "f"), self._chk(g, self.shape_p, "g"), int(nu)),
                "stokes_smooth")
        return u, p

    def smooth_f32(self, u, p, f, g, nu=1):
        """float32 smoothing steps of the mixed-precision inner cycle (float32 tensors)."""
        for t, sh, nm in ((u, self.shape_u, "u"), (p, self.shape_p, "p"), (f, self.shape_u, "f"), (g, self.shape_p, "g")):
            if t.dtype != torch.float32 or tuple(t.shape) != tuple(sh) or not t.is_contiguous() or t.device != self.device:
                raise ValueError("%s must be a contiguous float32 tensor of shape %s" % (nm, sh))
        B.check(self._lib.stokes_smooth_f32(self._h, _ptr(u), _ptr(p), _ptr(f), _ptr(g), int(nu)), "stokes_smooth_f32")
        return u, p

    def residual_restrict_f32(self, u, p, f, g):
        """float32 I^T (F - A x) from the finest level to the next (the inner cycle's transfer)."""
        for t, sh, nm in ((u, self.shape_u, "u"), (p, self.shape_p, "p"), (f, self.shape_u, "f"), (g, self.shape_p, "g")):
            if t.dtype != torch.float32 or tuple(t.shape) != tuple(sh) or not t.is_contiguous() or t.device != self.device:
                raise ValueError("%s must be a contiguous float32 tensor of shape %s" % (nm, sh))
        su, sp = self._coarse_shapes()
        fc = torch.zeros(su, dtype=torch.float32, device=self.device)
        gc = torch.zeros(sp, dtype=torch.float32, device=self.device)
        B.check(self._lib.stokes_residual_restrict_f32(self._h, _ptr(u), _ptr(p), _ptr(f), _ptr(g), _ptr(fc), _ptr(gc)),
                "stokes_residual_restrict_f32")
        return fc, gc

    def _coarse_shapes(self):
        nc = self.N // 2
        return (2, 2 * nc + 1, 2 * nc + 1), (nc + 1, nc + 1)

    def restrict(self, ru, rp):
        su, sp = self._coarse_shapes()
        fc = torch.zeros(su, dtype=torch.float64, device=self.device)
        gc = torch.zeros(sp, dtype=torch.float64, device=self.device)
        B.check(self._lib.stokes_restrict(self._h, self._chk(ru, self.shape_u, "ru"), self._chk(rp, self.shape_p, "rp"),
                                          _ptr(fc), _ptr(gc)), "stokes_restrict")
        return fc, gc

    def prolong_add(self, uc, pc, u, p):
        su, sp = self._coarse_shapes()
        B.check(self._lib.stokes_prolong_add(self._h, self._chk(uc, su, "uc"), self._chk(pc, sp, "pc"),
                                             self._chk(u, self.shape_u, "u"), self._chk(p, self.shape_p, "p")),
                "stokes_prolong_add")
        return u, p

    def autotune(self):
        """Time the float32 step variants on this solver's levels and keep the fastest per level."""
        B.check(self._lib.stokes_autotune(self._h), "stokes_autotune")

    def set_timing(self, enable=True):
        B.check(self._lib.stokes_set_timing(self._h, int(enable)), "stokes_set_timing")

    def timing(self):
        """(smoothing ms total, smoothing steps, residual ms total, residual launches) since set_timing."""
        sm, rm = ctypes.c_double(), ctypes.c_double()
        sc, rc = ctypes.c_longlong(), ctypes.c_longlong()
        B.check(self._lib.stokes_get_timing(self._h, ctypes.byref(sm), ctypes.byref(sc), ctypes.byref(rm),
                                            ctypes.byref(rc)), "stokes_get_timing")
        return sm.value, sc.value, rm.value, rc.value

    def timing_fused(self):
        """(ms total, steps) of the finest-level smoothing steps that also add the coarse-grid
        correction (the first post-smoothing step of a planar level) since set_timing."""
        ms, cnt = ctypes.c_double(), ctypes.c_longlong()
        B.check(self._lib.stokes_get_timing_fused(self._h, ctypes.byref(ms), ctypes.byref(cnt)),
                "stokes_get_timing_fused")
        return ms.value, cnt.value

    def kernel_launches(self):
        return int(self._lib.stokes_kernel_launches(self._h))

    def euler_rhs(self, u_prev, f_nodal, g_nodal):
        """Right-hand side (f, g) of one implicit Euler step with beta = 1/dt (stokes_euler_rhs):
        the load vectors of the nodal data f_nodal + beta u_prev and g_nodal (shifted to zero mean)."""
        f, g = self.zeros_u(), self.zeros_p()
        B.check(self._lib.stokes_euler_rhs(self._h, self._chk(u_prev, self.shape_u, "u_prev"),
                                           self._chk(f_nodal, self.shape_u, "f_nodal"),
                                           self._chk(g_nodal, self.shape_p, "g_nodal"), _ptr(f), _ptr(g)),
                "stokes_euler_rhs")
        return f, g

    def make_consistent(self, g):
        """g <- g - (sum g) M_P 1 in place (pressure right-hand side orthogonal to constants)."""
        B.check(self._lib.stokes_make_consistent(self._h, self._chk(g, self.shape_p, "g")), "stokes_make_consistent")
        return g

    def mass_apply(self, a):
        """M_U a for a velocity array (boundary entries of a count as given; rows on the boundary are 0)."""
        f, _ = self.load_vectors(a, self.zeros_p(), project_g=False)
        return f

    def mass_dot(self, a, b):
        out = ctypes.c_double()
        B.check(self._lib.stokes_mass_dot(self._h, self._chk(a, self.shape_u, "a"), self._chk(b, self.shape_u, "b"),
                                          ctypes.byref(out)), "stokes_mass_dot")
        return out.value


_TORCH_ALLOCATOR = None   # the registered callbacks (kept alive while registered)


def _torch_alloc(nbytes, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:
        return None


def _torch_free(ptr, nbytes, stream, ctx):
    torch.cuda.caching_allocator_delete(int(ptr))


def use_torch_allocator(enable=True):
    """Let PyTorch's caching allocator serve the device buffers of solvers set up from now on
    (stokes_set_allocator); enable=False restores cudaMalloc for later setups.  Solvers keep the
    allocator they were set up with."""
    global _TORCH_ALLOCATOR
    lib = B.load()
    if enable:
        cbs = (B.ALLOC_FN(_torch_alloc), B.FREE_FN(_torch_free))
        B.check(lib.stokes_set_allocator(cbs[0], cbs[1], None), "stokes_set_allocator")
        # earlier callbacks stay referenced by the solvers that use them
        _KEEP.append(cbs)
        _TORCH_ALLOCATOR = cbs
    else:
        B.check(lib.stokes_set_allocator(B.ALLOC_FN(), B.FREE_FN(), None), "stokes_set_allocator")
        _TORCH_ALLOCATOR = None


_KEEP = []


def step_variant(levels):
    """Float32 Uzawa step variant used for levels with N = 2^levels (0-3 fused tiles 32x16, 32x8,
    64x8, 16x16; 4-6 three-kernel step with blocks 32x8, 16x8, 8x8; 7-9 fused step on
    component-pair tiles, 28 cells wide; 10-11 fused step with the coefficients in registers)."""
    return int(B.load().stokes_step_variant(int(levels)))


def set_step_variant(levels, variant):
    """Forces the float32 Uzawa step variant for levels with N = 2^levels (process-wide; graphs
    captured earlier keep theirs)."""
    B.check(B.load().stokes_set_step_variant(int(levels), int(variant)), "stokes_set_step_variant")


def planar_step_variant(levels):
    """Step variant used for planar float32 levels with N = 2^levels (0 one tile per CTA; 1, 2
    persistent CTAs with two tile buffers, 8 or 16 warps)."""
    return int(B.load().stokes_planar_step_variant(int(levels)))


def set_planar_step_variant(levels, variant):
    """Forces the planar step variant for levels with N = 2^levels (process-wide)."""
    B.check(B.load().stokes_set_planar_step_variant(int(levels), int(variant)), "stokes_set_planar_step_variant")


class BatchSolver:
    """Many independent solves (levels, beta per instance) run to convergence in one CUDA-graph
    launch (stokes_batch_setup / stokes_batch_solve)."""

    def __init__(self, levels, betas, *, precision="mixed", nu_pre=3, nu_post=3, tau=0.8, sigma=0.8, gamma=1,
                 coarse_level=0, tma_level=0, coop_level=0, autotune=True, device=None):
        self._lib = B.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.levels = [int(l) for l in levels]
        self.betas = [float(b) for b in betas]
        assert len(self.levels) == len(self.betas) and len(self.levels) > 0
        prm = B.Params()
        self._lib.stokes_default_params(ctypes.byref(prm), 1, 0.0)
        prm.nu_pre, prm.nu_post, prm.tau, prm.sigma, prm.gamma = nu_pre, nu_post, tau, sigma, gamma
        prm.coarse_level = coarse_level
        prm.tma_level = tma_level
        prm.coop_level = coop_level
        prm.precision = _PREC[precision]
        n = len(self.levels)
        lv = (ctypes.c_int * n)(*self.levels)
        bt = (ctypes.c_double * n)(*self.betas)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream()
            B.check(self._lib.stokes_batch_setup(n, lv, bt, ctypes.byref(prm), ctypes.c_void_p(s.cuda_stream),
                                                 int(autotune), ctypes.byref(h)), "stokes_batch_setup")
        self._h = h
        self.count = n

    def shapes(self, i):
        N = 2 ** self.levels[i]
        return (2, 2 * N + 1, 2 * N + 1), (N + 1, N + 1)

    def solve(self, fs, gs, tol=1e-8, max_cycles=200, us=None, ps=None):
        n = self.count
        us = [torch.zeros(self.shapes(i)[0], dtype=torch.float64, device=self.device) for i in range(n)] \
            if us is None else us
        ps = [torch.zeros(self.shapes(i)[1], dtype=torch.float64, device=self.device) for i in range(n)] \
            if ps is None else ps
        for i in range(n):
            su, sp = self.shapes(i)
            for t, sh in ((us[i], su), (ps[i], sp), (fs[i], su), (gs[i], sp)):
                if t.dtype != torch.float64 or tuple(t.shape) != sh or not t.is_contiguous() or t.device != self.device:
                    raise ValueError("instance %d: expected contiguous float64 tensors of shape %s" % (i, sh))
        arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        cyc = (ctypes.c_int * n)()
        rel = (ctypes.c_double * n)()
        st = self._lib.stokes_batch_solve(self._h, arr(us), arr(ps), arr(fs), arr(gs), float(tol), int(max_cycles),
                                          cyc, rel)
        if st not in (B.OK, B.NOT_CONVERGED, B.DIVERGED):
            B.check(st, "stokes_batch_solve")
        return us, ps, list(cyc), list(rel), st

    def kernel_launches(self):
        return int(self._lib.stokes_batch_kernel_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stokes_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
