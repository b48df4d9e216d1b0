"""Alg. 2 (Clenshaw) applied to a sparse Hermitian matrix and a dense block.

TEST INFRASTRUCTURE (see ``oracle/__init__``).  FP64 / complex128 throughout;
the sparse product is scipy's CSR times dense, used as a library step.
"""
from __future__ import annotations

import numpy as np


def clenshaw_apply(A, a: np.ndarray, l1: float, l2: float, X: np.ndarray) -> np.ndarray:
    """V = rho(l(A)) X with rho(x) = sum_{j=0}^{k} a_j T_j(x), k = len(a) - 1 (Alg. 2).

    A is a scipy sparse matrix, X an n x p array.  The steps follow Alg. 2 in
    order, with the Y, W, V names and the swaps of the paper.  The first step
    uses the division-free form V = 2 l1 A W + 2 l2 W + a_{k-1} Y with
    W = a_k Y, equal to the printed (2 l2 + a_{k-1}/a_k) W when a_k != 0.
    Degrees 0 and 1 reduce to a_0 Y and l(A)(a_1 Y) + a_0 Y.
    """
    k = len(a) - 1
    Y = np.array(X, copy=True)
    if k == 0:
        return a[0] * Y
    W = a[k] * Y
    if k == 1:
        return l1 * (A @ W) + l2 * W + a[0] * Y
    V = 2.0 * l1 * (A @ W) + 2.0 * l2 * W + a[k - 1] * Y
    V, W = W, V
    for j in range(k - 2, 0, -1):
        V = 2.0 * l1 * (A @ W) + 2.0 * l2 * W - V + a[j] * Y
        V, W = W, V
    return l1 * (A @ W) + l2 * W - V + a[0] * Y


def filter_dense_definition(Adense: np.ndarray, a: np.ndarray, l1: float, l2: float,
                            X: np.ndarray) -> np.ndarray:
    """rho(l(A)) X by definition: U diag(rho(l(lambda))) U^H X with A = U diag(lambda) U^H.

    rho(l(lambda)) = sum_j a_j cos(j arccos(l(lambda))) evaluated directly; needs
    the spectrum of l(A) inside [-1, 1].  Dense, for small n only.
    """
    lam, U = np.linalg.eigh(Adense)
    x = np.clip(l1 * lam + l2, -1.0, 1.0)
    th = np.arccos(x)
    r = np.zeros_like(lam)
    for j in range(len(a)):
        r = r + a[j] * np.cos(j * th)
    return U @ (r[:, None] * (U.conj().T @ X))
