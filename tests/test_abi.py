"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point that
include/stokes_mg.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(stokes_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1502_04070_gb300 import _binding, build
    build.build()
    lib = _binding.load()
    names = declared_functions()
    assert len(names) >= 15
    for nm in sorted(names):
        assert hasattr(lib, nm), nm
        assert nm in _binding.SIGNATURES, "binding lacks " + nm


def test_status_strings_and_defaults_without_gpu():
    from paper_1502_04070_gb300 import _binding
    lib = _binding.load()
    assert lib.stokes_status_str(0) == b"ok"
    assert lib.stokes_status_str(5) == b"diverged"
    prm = _binding.Params()
    lib.stokes_default_params(ctypes.byref(prm), 5, 1.0)
    assert (prm.nu_pre, prm.nu_post, prm.tau, prm.sigma, prm.gamma) == (3, 3, 0.8, 0.8, 1)


def test_setup_rejects_bad_arguments_without_touching_the_gpu():
    from paper_1502_04070_gb300 import _binding
    lib = _binding.load()
    h = ctypes.c_void_p()
    prm = _binding.Params()
    lib.stokes_default_params(ctypes.byref(prm), 0, 1.0)        # levels < 1
    assert lib.stokes_setup(ctypes.byref(prm), None, ctypes.byref(h)) == _binding.ERR_BAD_ARG
    lib.stokes_default_params(ctypes.byref(prm), 4, -1.0)       # beta < 0
    assert lib.stokes_setup(ctypes.byref(prm), None, ctypes.byref(h)) == _binding.ERR_BAD_ARG
    lib.stokes_default_params(ctypes.byref(prm), 4, float("nan"))
    assert lib.stokes_setup(ctypes.byref(prm), None, ctypes.byref(h)) == _binding.ERR_BAD_ARG
    assert lib.stokes_setup(None, None, ctypes.byref(h)) == _binding.ERR_BAD_ARG
    for levels, c in ((3, 3), (6, 4), (6, -1)):                 # coarsest level out of range
        lib.stokes_default_params(ctypes.byref(prm), levels, 1.0)
        prm.coarse_level = c
        assert lib.stokes_setup(ctypes.byref(prm), None, ctypes.byref(h)) == _binding.ERR_BAD_ARG
    for t in (-1, 1, 4):                                           # planar float32 levels start at 5
        lib.stokes_default_params(ctypes.byref(prm), 6, 1.0)
        prm.precision, prm.tma_level = _binding.MIXED, t
        assert lib.stokes_setup(ctypes.byref(prm), None, ctypes.byref(h)) == _binding.ERR_BAD_ARG, t
    # the L-shaped domain needs Uzawa cycles with coarsest level 1
    for field, value in (("coarse_level", 0), ("coarse_level", 2), ("smoother", _binding.NORMAL_EQ), ("domain", 2)):
        lib.stokes_default_params(ctypes.byref(prm), 5, 1.0)
        prm.domain, prm.coarse_level = _binding.L_SHAPE, 1
        setattr(prm, field, value)
        assert lib.stokes_setup(ctypes.byref(prm), None, ctypes.byref(h)) == _binding.ERR_BAD_ARG, field


def test_entry_points_reject_null_handles_without_touching_the_gpu():
    from paper_1502_04070_gb300 import _binding
    lib = _binding.load()
    buf = ctypes.c_void_p(16)       # never dereferenced: the null handle is rejected first
    assert lib.stokes_euler_rhs(None, buf, buf, buf, buf, buf) == _binding.ERR_BAD_ARG
    assert lib.stokes_load_vectors(None, buf, buf, 1, buf, buf) == _binding.ERR_BAD_ARG
    assert lib.stokes_cycle(None, buf, buf, buf, buf) == _binding.ERR_BAD_ARG


def test_step_variant_selection_without_gpu():
    """The variant table is host state: out-of-range sizes and variants are rejected, a valid
    choice reads back."""
    from paper_1502_04070_gb300 import _binding
    lib = _binding.load()
    assert lib.stokes_set_step_variant(1, 0) == _binding.ERR_BAD_ARG
    assert lib.stokes_set_step_variant(32, 0) == _binding.ERR_BAD_ARG
    assert lib.stokes_set_step_variant(5, 12) == _binding.ERR_BAD_ARG
    assert lib.stokes_set_step_variant(5, -1) == _binding.ERR_BAD_ARG
    assert lib.stokes_set_planar_step_variant(5, 6) == _binding.ERR_BAD_ARG
    assert lib.stokes_set_planar_step_variant(1, 0) == _binding.ERR_BAD_ARG
    assert lib.stokes_planar_step_variant(40) == -1
    assert lib.stokes_step_variant(1) == -1
    old = lib.stokes_step_variant(5)
    assert lib.stokes_set_step_variant(5, 6) == _binding.OK
    assert lib.stokes_step_variant(5) == 6
    assert lib.stokes_set_step_variant(5, old) == _binding.OK


def test_allocator_registration_without_gpu():
    """stokes_set_allocator takes both callbacks or neither (cudaMalloc again)."""
    from paper_1502_04070_gb300 import _binding as B
    lib = B.load()
    keep = B.ALLOC_FN(lambda nbytes, stream, ctx: None)
    assert lib.stokes_set_allocator(keep, B.FREE_FN(), None) == B.ERR_BAD_ARG
    assert lib.stokes_set_allocator(B.ALLOC_FN(), B.FREE_FN(), None) == B.OK


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_1502_04070_gb300 import _binding
    saved = _binding._lib
    try:
        _binding._lib = None
        with pytest.raises(RuntimeError):
            _binding.load(str(tmp_path / "missing.so"))
    finally:
        _binding._lib = saved


def test_time_stepper_rejects_bad_step_without_gpu():
    from paper_1502_04070_gb300.timestep import ImplicitEuler
    for dt in (0.0, -1e-3, float("nan")):
        with pytest.raises(ValueError):
            ImplicitEuler(4, dt)


def test_every_entry_point_rejects_bad_arguments_before_device_work():
    """Failure handling (every call returns a status, nothing aborts): each entry point that takes a
    handle rejects a null handle, and the handle-free ones reject out-of-range sizes, before any
    CUDA call; destroy and the launch counters accept null."""
    from paper_1502_04070_gb300 import _binding as B
    lib = B.load()
    buf = ctypes.c_void_p(16)                  # never dereferenced
    d = ctypes.c_double()
    bad = B.ERR_BAD_ARG
    calls = {
        "stokes_autotune": (None,),
        "stokes_set_beta": (None, 1.0),
        "stokes_sizes": (None, None, None, None, None),
        "stokes_cycle": (None, buf, buf, buf, buf),
        "stokes_solve": (None, buf, buf, buf, buf, 1e-8, 10, None, None),
        "stokes_residual": (None, buf, buf, buf, buf, buf, buf),
        "stokes_residual_norm": (None, buf, buf, buf, buf, ctypes.byref(d)),
        "stokes_smooth": (None, buf, buf, buf, buf, 1),
        "stokes_smooth_f32": (None, buf, buf, buf, buf, 1),
        "stokes_restrict": (None, buf, buf, buf, buf),
        "stokes_prolong_add": (None, buf, buf, buf, buf),
        "stokes_load_vectors": (None, buf, buf, 1, buf, buf),
        "stokes_euler_rhs": (None, buf, buf, buf, buf, buf),
        "stokes_make_consistent": (None, buf),
        "stokes_mass_dot": (None, buf, buf, ctypes.byref(d)),
        "stokes_set_timing": (None, 1),
        "stokes_get_timing": (None, None, None, None, None),
        "stokes_get_timing_fused": (None, None, None),
        "stokes_residual_norm2_noalloc": (0, 1.0, buf, buf, buf, buf, ctypes.byref(d), None),
        "stokes_batch_solve": (None, None, None, None, None, 1e-8, 10, None, None),
        "stokes_transfer_weights": (None,),
        "stokes_embed_weights": (None,),
        "stokes_coarse_inverse": (0.0, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == bad, name
    assert lib.stokes_residual_norm2_noalloc(30, 1.0, buf, buf, buf, buf, ctypes.byref(d), None) == bad
    n = ctypes.c_int(1)
    lv = (ctypes.c_int * 1)(3)
    be = (ctypes.c_double * 1)(1.0)
    out = ctypes.c_void_p()
    prm = B.Params()
    lib.stokes_default_params(ctypes.byref(prm), 3, 1.0)
    assert lib.stokes_batch_setup(0, lv, be, ctypes.byref(prm), None, 0, ctypes.byref(out)) == bad
    assert lib.stokes_batch_setup(n.value, None, be, ctypes.byref(prm), None, 0, ctypes.byref(out)) == bad
    lib.stokes_destroy(None)
    lib.stokes_batch_destroy(None)
    assert lib.stokes_kernel_launches(None) == 0
    assert lib.stokes_batch_kernel_launches(None) == 0


def test_header_is_plain_c():
    """include/stokes_mg.h is a C-ABI header: it compiles as C99 (no C++ or torch types)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            r = subprocess.run([cc, "-fsyntax-only", "-std=c99", "-Wall", "-Werror", "-x", "c",
                                os.path.join(ROOT, "include", fn)], capture_output=True, text=True)
            assert r.returncode == 0, r.stderr
