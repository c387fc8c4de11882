"""ctypes declarations of the C-ABI in include/stokes_mg.h (argument marshalling only).

The library is loaded from the package's in-tree build directory; there is no fallback: if it is
missing or fails to load, every call raises.
"""
import ctypes
import os

from . import build as _build

OK, ERR_BAD_ARG, ERR_OOM, ERR_CUDA, NOT_CONVERGED, DIVERGED, ERR_TIMEOUT = range(7)
UZAWA, NORMAL_EQ = 0, 1
UNIT_SQUARE, L_SHAPE = 0, 1
FP64, MIXED = 0, 1


class Params(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("smoother", ctypes.c_int),
        ("gamma", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("inner_cycles", ctypes.c_int),
        ("coarse_level", ctypes.c_int),
        ("domain", ctypes.c_int),
        ("tma_level", ctypes.c_int),
        ("coop_level", ctypes.c_int),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("cycles", ctypes.c_int),
        ("rel_residual", ctypes.c_double),
        ("mean_rate", ctypes.c_double),
        ("initial_residual", ctypes.c_double),
        ("rhs_norm", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SZ = ctypes.c_size_t

# stokes_alloc_fn / stokes_free_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

# name -> (restype, argtypes); every symbol declared in include/stokes_mg.h
SIGNATURES = {
    "stokes_default_params": (None, [ctypes.POINTER(Params), _I, _D]),
    "stokes_setup": (_I, [ctypes.POINTER(Params), _P, ctypes.POINTER(_P)]),
    "stokes_set_allocator": (_I, [ALLOC_FN, FREE_FN, _P]),
    "stokes_set_beta": (_I, [_P, _D]),
    "stokes_destroy": (None, [_P]),
    "stokes_status_str": (ctypes.c_char_p, [_I]),
    "stokes_sizes": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "stokes_cycle": (_I, [_P, _P, _P, _P, _P]),
    "stokes_solve": (_I, [_P, _P, _P, _P, _P, _D, _I, ctypes.POINTER(Report), ctypes.POINTER(_D)]),
    "stokes_residual": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "stokes_residual_norm": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(_D)]),
    "stokes_smooth": (_I, [_P, _P, _P, _P, _P, _I]),
    "stokes_smooth_f32": (_I, [_P, _P, _P, _P, _P, _I]),
    "stokes_residual_restrict_f32": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "stokes_restrict": (_I, [_P, _P, _P, _P, _P]),
    "stokes_prolong_add": (_I, [_P, _P, _P, _P, _P]),
    "stokes_load_vectors": (_I, [_P, _P, _P, _I, _P, _P]),
    "stokes_mass_dot": (_I, [_P, _P, _P, ctypes.POINTER(_D)]),
    "stokes_make_consistent": (_I, [_P, _P]),
    "stokes_euler_rhs": (_I, [_P, _P, _P, _P, _P, _P]),
    "stokes_transfer_weights": (_I, [_P]),
    "stokes_lshape_vertex_rows": (_I, [_I, _I, _P, _P, ctypes.POINTER(_D)]),
    "stokes_lshape_schur": (_I, [_I, _D, _P, _P, _P]),
    "stokes_lshape_coarse_inverse": (_I, [_D, _P, ctypes.POINTER(_I)]),
    "stokes_coarse_inverse": (_I, [_D, _P]),
    "stokes_stencil_class": (_I, [_I, _I, _I, ctypes.POINTER(_I)]),
    "stokes_stencil_rows": (_I, [_I, _D, _I, _P, _P, _P, _P, _P, _P]),
    "stokes_residual_norm2_noalloc": (_I, [_I, _D, _P, _P, _P, _P, _P, _P]),
    "stokes_batch_setup": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(Params), _P, _I,
                                ctypes.POINTER(_P)]),
    "stokes_batch_solve": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "stokes_batch_destroy": (None, [_P]),
    "stokes_euler_run": (_I, [_P, _P, _P, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _D, _I, ctypes.POINTER(_I),
                              ctypes.POINTER(_D)]),
    "stokes_batch_euler_run": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                    _I, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "stokes_batch_kernel_launches": (ctypes.c_ulonglong, [_P]),
    "stokes_autotune": (_I, [_P]),
    "stokes_step_variant": (_I, [_I]),
    "stokes_set_step_variant": (_I, [_I, _I]),
    "stokes_planar_step_variant": (_I, [_I]),
    "stokes_set_planar_step_variant": (_I, [_I, _I]),
    "stokes_step_tables_match": (_I, [_I, _D]),
    "stokes_set_timing": (_I, [_P, _I]),
    "stokes_get_timing": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                               ctypes.POINTER(ctypes.c_longlong)]),
    "stokes_get_timing_fused": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)]),
    "stokes_embed_weights": (_I, [_P]),
    "stokes_kernel_launches": (ctypes.c_ulonglong, [_P]),
}

_lib = None


def load(path: str = None):
    """Load (once) and return the CUDA library with typed entry points."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.library_path()
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is not built; run __graft_entry__.build() "
                           "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class StokesError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = load().stokes_status_str(status).decode()
        super().__init__("%s failed: %s (status %d)" % (what, msg, status))


def check(status, what):
    if status != OK:
        raise StokesError(status, what)
    return status
