"""The result by definition, for small matrices (oracle level O1).

TEST INFRASTRUCTURE (see ``oracle/__init__``).  The interior eigenproblem of
Sec. 1, Eq. (ori_problem): all (lambda_j, v_j) of the Hermitian A with
lambda_j in [a, b].  Dense LAPACK routines serve as library steps.
"""
from __future__ import annotations

import numpy as np


def interior_eigenpairs(Adense: np.ndarray, a: float, b: float):
    """All eigenpairs with a <= lambda <= b, ascending (Eq. (ori_problem))."""
    lam, U = np.linalg.eigh(Adense)
    sel = (lam >= a) & (lam <= b)
    return lam[sel], U[:, sel]


def all_eigenvalues(Adense: np.ndarray) -> np.ndarray:
    return np.linalg.eigvalsh(Adense)


def inertia_count_below(Adense: np.ndarray, sigma: float) -> int:
    """Number of eigenvalues of A below sigma, by Sylvester's law of inertia.

    A - sigma I = L D L^H (Bunch-Kaufman, scipy.linalg.ldl); A - sigma I and
    the block-diagonal D are congruent, so they have the same number of
    negative eigenvalues.  D has 1x1 and 2x2 blocks; its eigenvalues are
    counted directly.  Independent of the eigendecomposition above.
    """
    import scipy.linalg as sl
    n = Adense.shape[0]
    M = Adense - sigma * np.eye(n)
    _, D, _ = sl.ldl(M, lower=True, hermitian=True)
    neg = 0
    i = 0
    while i < n:
        if i + 1 < n and D[i + 1, i] != 0:
            blk = D[i:i + 2, i:i + 2]
            neg += int(np.sum(np.linalg.eigvalsh(blk) < 0))
            i += 2
        else:
            neg += int(D[i, i].real < 0)
            i += 1
    return neg


def interval_count(Adense: np.ndarray, a: float, b: float) -> int:
    """Eigenvalues in [a, b] from two inertia counts (a, b not eigenvalues)."""
    return inertia_count_below(Adense, b) - inertia_count_below(Adense, a)
