"""Helpers shared by the GPU tests: device copies and the derived tolerances."""
import numpy as np

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def empty_like_np(shape, is_complex):
    import torch
    return torch.zeros(shape, dtype=torch.complex128 if is_complex else torch.float64, device="cuda")


def clenshaw_tol(coef, X, eps):
    """Error bound used for Alg. 2 parity: the recurrence runs k steps, each
    adding a rounding error of order eps times the largest intermediate, and
    the Clenshaw intermediates are bounded by sum |a_j| times ||X||_max; a
    factor 50 covers the row length of the sparse products."""
    k = len(coef) - 1
    return 50.0 * max(k, 1) * eps * max(1.0, float(np.sum(np.abs(coef)))) * float(np.max(np.abs(X)))
