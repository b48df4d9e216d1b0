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
    """Error bound used for Alg. 2 parity.  The recurrence runs k steps; each
    adds a rounding error of order eps times the Clenshaw intermediates, which
    the filter keeps near sum |a_j| max|X|, and errors of independent sign add
    like a random walk: sqrt(k) eps sum|a_j| max|X|, with a margin of 4.
    tests/test_tolerances.py checks that an FP32 evaluation in another
    summation order stays well inside this bound, and that dropping any one
    a_j T_j term, the smallest plausible slip in the recurrence, exceeds it."""
    k = len(coef) - 1
    return 4.0 * np.sqrt(max(k, 1)) * eps * max(1.0, float(np.sum(np.abs(coef)))) * float(np.max(np.abs(X)))
