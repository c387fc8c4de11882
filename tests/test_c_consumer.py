"""A plain C program uses the C-ABI: it includes include/stokes_mg.h, links libstokes_mg.so and calls
the host-only entry points (defaults, status strings, a stencil class, the embedding weights, the
level-0 inverse, an argument error), with no GPU needed; its output is checked against the
library's Python binding and the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "stokes_mg.h"

int main(void) {
    stokes_params prm;
    double w[450], inv[729];
    int cls = -1;
    stokes_default_params(&prm, 5, 2.5);
    printf("params %d %d %.17g %.17g %d\n", prm.nu_pre, prm.nu_post, prm.tau, prm.sigma, prm.gamma);
    printf("status %s\n", stokes_status_str(STOKES_OK));
    if (stokes_stencil_class(4, 8, 3, &cls) != STOKES_OK) return 1;
    printf("class %d\n", cls);
    if (stokes_transfer_weights(w) != STOKES_OK) return 2;
    printf("weight %.17g %.17g\n", w[0], w[1 * 225 + 4 * 25 + 2 * 5 + 2]);
    if (stokes_coarse_inverse(1.0, inv) != STOKES_OK) return 3;
    printf("inv %.17g %.17g\n", inv[0], inv[26 * 27 + 26]);
    printf("bad %d\n", (int)stokes_cycle(0, 0, 0, 0, 0));
    return 0;
}
"""


def test_c_program_links_and_calls_the_library(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1502_04070_gb300 import _binding
    from paper_1502_04070_gb300 import build as b
    lib = _binding.load()
    libdir = os.path.dirname(b.library_path())
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", str(src), "-I", os.path.join(ROOT, "include"),
                        "-L", libdir, "-lstokes_mg", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.stdout, r.stderr)
    out = {ln.split()[0]: ln.split()[1:] for ln in r.stdout.strip().splitlines()}
    assert out["params"][:2] == ["3", "3"] and float(out["params"][2]) == 0.8 and out["params"][4] == "1"
    assert out["status"] == [lib.stokes_status_str(0).decode()]
    # cell (8, 3) of N = 16 lies on the mid-line x = 1/2 below the centre: class 2
    assert out["class"] == ["2"]
    w = np.zeros(450)
    lib.stokes_transfer_weights(w.ctypes.data_as(_binding.ctypes.c_void_p))
    assert float(out["weight"][0]) == w[0] and float(out["weight"][1]) == w[225 + 100 + 10 + 2]
    from oracle import fem
    from oracle import multigrid as mg
    H = mg.Hierarchy(1, 1.0, fem.discretizations(1))
    ref = np.linalg.inv(H.coarse_bordered)[:27, :27]
    assert abs(float(out["inv"][0]) - ref[0, 0]) <= 1e-10 * np.abs(ref).max()
    assert abs(float(out["inv"][1]) - ref[26, 26]) <= 1e-10 * np.abs(ref).max()
    assert int(out["bad"][0]) == _binding.ERR_BAD_ARG
