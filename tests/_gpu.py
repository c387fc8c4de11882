"""Helpers shared by the GPU tests (lattice arrays <-> torch, oracle hierarchies)."""
import numpy as np
import torch


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64))).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale
