"""GB300 coupled multigrid solver for the generalized Stokes system (Taylor-Hood P2-P1).

Robust multigrid with an Uzawa-type smoother (Takacs, SINUM 53(6), 2015), hand-written CUDA for
sm_103a behind a C-ABI (include/stokes_mg.h).  Importing the package does not load the CUDA
library; the first solver construction does, and fails loudly if it is missing.
"""
__all__ = ["Solver", "workloads"]


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver
        return Solver
    raise AttributeError(name)
