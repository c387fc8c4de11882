"""Seeded synthetic inputs for the generalized Stokes solver.

This module only draws numbers and evaluates the problem data (right-hand-side functions); it holds
none of the method's arithmetic (no matrices, no smoothing, no transfers).  Both the CUDA path and
the CPU oracle are fed from here.

Layouts (canonical, row-major, y outer / x inner):
    velocity nodal values  (2, 2N+1, 2N+1)   on the full P2 lattice of spacing 1/(2N)
    pressure nodal values  (N+1, N+1)        on the vertex lattice of spacing 1/N
with N = 2^(k+1) on grid level k (the unit square split into 8 triangles on level 0 and refined
uniformly k times).  The mesh leg is h = 1/N, so "h = 1/32" is level k = 4.
"""
import math

import numpy as np


def level_of_h(inv_h: int) -> int:
    """Grid level k with leg h = 1/inv_h (N = 2^(k+1) = inv_h)."""
    k = int(round(math.log2(inv_h))) - 1
    assert 2 ** (k + 1) == inv_h and k >= 0
    return k


def sizes(k: int):
    n = 2 ** (k + 1)
    return n, 2 * n + 1, n + 1


def dofs(k: int) -> int:
    """Unknowns on level k: 2 (2N-1)^2 interior velocity values + (N+1)^2 pressure values."""
    n = 2 ** (k + 1)
    return 2 * (2 * n - 1) ** 2 + (n + 1) ** 2


def random_nodal(k: int, seed: int, with_g: bool = True, rng=None):
    """f with i.i.d. uniform[-1, 1] nodal values (boundary values set to zero), and g likewise
    (all vertices) or zero.  Drawn in the order: f_x, f_y, g, each row-major."""
    n, m2, m1 = sizes(k)
    rng = np.random.default_rng(seed) if rng is None else rng
    f = rng.uniform(-1.0, 1.0, size=(2, m2, m2))
    f[:, 0, :] = 0.0
    f[:, -1, :] = 0.0
    f[:, :, 0] = 0.0
    f[:, :, -1] = 0.0
    g = rng.uniform(-1.0, 1.0, size=(m1, m1)) if with_g else np.zeros((m1, m1))
    return f, g


def random_state(k: int, seed: int):
    """A random iterate (u, p): uniform[-1, 1] with u = 0 on the boundary lattice points."""
    f, g = random_nodal(k, seed, with_g=True)
    return f, g


# ------------------------------------------------------------------ manufactured solution
# u = curl psi = (d_y psi, -d_x psi), psi = sin^2(pi x) sin^2(pi y);  p = cos(pi x) cos(pi y).
# u vanishes on the boundary, div u = 0, int p = 0.  f = -Lap u + beta u + grad p (strong form).

def exact_u(x, y):
    pi = math.pi
    ux = pi * np.sin(pi * x) ** 2 * np.sin(2 * pi * y)
    uy = -pi * np.sin(2 * pi * x) * np.sin(pi * y) ** 2
    return ux, uy


def exact_grad_u(x, y):
    """((d_x ux, d_y ux), (d_x uy, d_y uy))."""
    pi = math.pi
    dxux = pi * pi * np.sin(2 * pi * x) * np.sin(2 * pi * y)
    dyux = 2 * pi * pi * np.sin(pi * x) ** 2 * np.cos(2 * pi * y)
    dxuy = -2 * pi * pi * np.cos(2 * pi * x) * np.sin(pi * y) ** 2
    dyuy = -pi * pi * np.sin(2 * pi * x) * np.sin(2 * pi * y)
    return (dxux, dyux), (dxuy, dyuy)


def exact_p(x, y):
    return np.cos(math.pi * x) * np.cos(math.pi * y)


def manufactured_f(x, y, beta):
    pi = math.pi
    ux, uy = exact_u(x, y)
    lap_ux = pi * (2 * pi * pi * np.cos(2 * pi * x) * np.sin(2 * pi * y)
                   - 4 * pi * pi * np.sin(pi * x) ** 2 * np.sin(2 * pi * y))
    lap_uy = -pi * (2 * pi * pi * np.sin(2 * pi * x) * np.cos(2 * pi * y)
                    - 4 * pi * pi * np.sin(2 * pi * x) * np.sin(pi * y) ** 2)
    dpx = -pi * np.sin(pi * x) * np.cos(pi * y)
    dpy = -pi * np.cos(pi * x) * np.sin(pi * y)
    return -lap_ux + beta * ux + dpx, -lap_uy + beta * uy + dpy


def manufactured_nodal(k: int, beta: float):
    """Nodal values of f (full P2 lattice, boundary included) and g = 0 for the manufactured
    solution above."""
    n, m2, m1 = sizes(k)
    t = np.arange(m2) / (2.0 * n)
    X, Y = np.meshgrid(t, t)          # Y varies along rows
    fx, fy = manufactured_f(X, Y, beta)
    return np.stack([fx, fy]), np.zeros((m1, m1))


# ------------------------------------------------------------------ batches
def batch_spec(n_inst: int, seed: int, k_min: int = 4, k_max: int = 8,
               beta_lo: float = 1e-2, beta_hi: float = 1e8):
    """Levels uniform in {k_min..k_max} and beta log-uniform in [beta_lo, beta_hi]."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(k_min, k_max + 1, size=n_inst)
    betas = np.exp(rng.uniform(math.log(beta_lo), math.log(beta_hi), size=n_inst))
    seeds = rng.integers(0, 2 ** 31 - 1, size=n_inst)
    return [int(k) for k in ks], [float(b) for b in betas], [int(s) for s in seeds]
