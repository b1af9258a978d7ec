"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

from oracle import discretization as disc

STENCIL = disc.STENCIL


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def j_to_dev(J):
    return [dev(J[s]) for s in STENCIL]


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)
