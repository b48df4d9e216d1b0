"""AdaPolySI (Alg. 4) step by step, in FP64 on the CPU (oracle level O2).

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Every step follows the paper
in its order and notation.  Library steps: scipy sparse times dense, numpy
Cholesky / triangular solve / eigh.  Random draws (the initial block V^(0) and
the Lanczos start vector) are inputs, not drawn here.

Readings taken where the paper is silent or ambiguous:

* The Lanczos bounds (Sec. 3.4, "a few iterations") run ``lanczos_steps``
  steps with full reorthogonalisation; lambda_max is padded outward to
  theta_max + |beta_m s_m| + pad (theta_max - theta_min), lambda_min likewise,
  and the two are clipped to the Gershgorin interval, which always holds the
  spectrum.
* The orthogonalisation of Alg. 4, orth([V, X]): X is projected against the locked V twice
  (block classical Gram-Schmidt), then orthonormalised by Cholesky QR twice
  (CholQR2).  Q^(i) is read as the new part, orthogonal to V.
* When the first Cholesky factorisation of CholQR2 meets a non-positive pivot,
  the shifted Cholesky QR of Fukaya et al. (SIAM J. Sci. Comput. 2020) with
  shift 11 (n p + p (p + 1)) u ||X||_F^2 runs first (CholQR3).
* Locking uses ||r_j|| <= tau_c ||A||, the convergence test of Sec. 4, with
  ||A|| = max(|theta_min|, |theta_max|) from the Lanczos Ritz values: they lie
  inside the spectrum, so this never exceeds the true spectral radius and a
  locked pair satisfies ||r_j|| <= tau_c ||A|| for the true ||A|| (the padded
  bounds lmin, lmax, which contain the spectrum, serve the map l only).
* n_check^(i-1) is the value from the last iteration that computed it (0 at
  the start); iterations with e^(i) = 0 leave it and the degree unchanged.
* The loop stops after ``max_iter`` iterations with status "no_convergence"
  and the pairs locked so far.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import chebyshev as cb
from .filter import clenshaw_apply


@dataclass
class Params:
    p: int
    k_fixed: int = 0            # 0: adaptive (Eq. (compute_k_1) + Alg. 3); > 0: fixed degree
    C: float = 1.4              # Eq. (compute_k_1)
    k_ratio: float = 2.5        # k = ceil(2.5 k^(1)) (Sec. 4)
    damping: str = cb.DAMP_LANCZOS_M
    m: float = 0.5              # damping exponent (Sec. 4)
    tau_a: float = 1e-3         # adaptive threshold (Sec. 3.1, Sec. 4)
    tau_c: float = 1e-10        # convergence threshold (Sec. 4)
    max_iter: int = 50
    lanczos_steps: int = 40
    bound_pad: float = 0.01
    spurious_rule: bool = True  # spurious-eigenvalue test of Alg. 4 (Sec. 3.3.2)
    locking: bool = True        # implicit deflation (Sec. 3.3.3)


@dataclass
class Result:
    eigvals: np.ndarray
    eigvecs: np.ndarray
    residuals: np.ndarray       # ||A v - lambda v|| / ||A||
    status: str
    stats: dict = field(default_factory=dict)


# --- Sec. 3.4: spectrum bounds ----------------------------------------------------

def gershgorin(A):
    """[min_i (Re a_ii - r_i), max_i (Re a_ii + r_i)], r_i = sum_{j != i} |a_ij|."""
    d = A.diagonal()
    r = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    return float(np.min(d.real - r)), float(np.max(d.real + r))


def lanczos_bounds(A, steps: int, v0: np.ndarray, pad: float = 0.01):
    """Estimate [lambda_min, lambda_max] by Lanczos with full reorthogonalisation.

    Returns (lmin, lmax, info) following the padding rule in the module notes.
    """
    n = A.shape[0]
    m = min(steps, n)
    q = v0 / np.linalg.norm(v0)
    Q = [q]
    alphas, betas = [], []
    for j in range(m):
        w = A @ Q[j]
        alpha = float(np.real(np.vdot(Q[j], w)))
        w = w - alpha * Q[j]
        if j > 0:
            w = w - betas[j - 1] * Q[j - 1]
        Qm = np.stack(Q, axis=1)
        for _ in range(2):
            w = w - Qm @ (Qm.conj().T @ w)
        beta = float(np.linalg.norm(w))
        alphas.append(alpha)
        betas.append(beta)
        if j == m - 1 or beta <= 1e-14 * max(1.0, max(abs(x) for x in alphas)):
            break
        Q.append(w / beta)
    mm = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:mm - 1], 1) + np.diag(betas[:mm - 1], -1)
    theta, S = np.linalg.eigh(T)
    res_lo = abs(betas[-1] * S[-1, 0])
    res_hi = abs(betas[-1] * S[-1, -1])
    spread = theta[-1] - theta[0]
    lmax = theta[-1] + res_hi + pad * spread
    lmin = theta[0] - res_lo - pad * spread
    g_lo, g_hi = gershgorin(A)
    lmax = min(lmax, g_hi)
    lmin = max(lmin, g_lo)
    return lmin, lmax, dict(theta_min=theta[0], theta_max=theta[-1], steps=mm,
                            res_lo=res_lo, res_hi=res_hi, gersh=(g_lo, g_hi))


# --- Alg. 4, orthogonalisation ------------------------------------------------

def cholqr(X: np.ndarray):
    """One Cholesky QR: G = X^H X = R^H R, Q = X R^{-1}.  Raises LinAlgError
    on a non-positive pivot."""
    import scipy.linalg as sl
    G = X.conj().T @ X
    G = 0.5 * (G + G.conj().T)
    R = np.linalg.cholesky(G).conj().T
    Q = sl.solve_triangular(R.T, X.T, lower=True).T      # Q R = X  <=>  R^T Q^T = X^T
    return Q, R


def shifted_cholqr(X: np.ndarray):
    import scipy.linalg as sl
    n, p = X.shape
    u = np.finfo(np.float64).eps / 2
    s = 11.0 * (n * p + p * (p + 1)) * u * np.linalg.norm(X) ** 2
    G = X.conj().T @ X
    G = 0.5 * (G + G.conj().T) + s * np.eye(p)
    R = np.linalg.cholesky(G).conj().T
    Q = sl.solve_triangular(R.T, X.T, lower=True).T
    return Q, R


def cholqr2(X: np.ndarray):
    """CholQR2 (with a shifted first pass when plain Cholesky breaks down)."""
    try:
        Q1, _ = cholqr(X)
    except np.linalg.LinAlgError:
        Q1, _ = shifted_cholqr(X)
        Q1, _ = cholqr(Q1)
    Q, _ = cholqr(Q1)
    return Q


def project_out(V: np.ndarray, X: np.ndarray) -> np.ndarray:
    """X - V (V^H X), twice (block classical Gram-Schmidt against locked V)."""
    if V.shape[1] == 0:
        return X
    for _ in range(2):
        X = X - V @ (V.conj().T @ X)
    return X


# --- Alg. 1: Rayleigh-Ritz ------------------------------------------------------------

def rayleigh_ritz(A, Q: np.ndarray):
    """B = Q^H A Q, B = U Lambda U^H, V = Q U (Alg. 1, function Rayleigh-Ritz)."""
    AQ = A @ Q
    B = Q.conj().T @ AQ
    B = 0.5 * (B + B.conj().T)
    lam, U = np.linalg.eigh(B)
    return lam, Q @ U


def residual_norms(A, V: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """||A v_j - lambda_j v_j||_2 for each column (residual step of Alg. 4)."""
    R = A @ V - V * lam[None, :]
    return np.linalg.norm(R, axis=0)


# --- Eq. (tau_s) -------------------------------------------------------------------

def tau_s(lam_in: np.ndarray, a: float, b: float) -> float:
    """tau_s = min_j min(|lambda_j - a|, |lambda_j - b|) over in-interval Ritz values."""
    return float(np.min(np.minimum(np.abs(lam_in - a), np.abs(lam_in - b))))


# --- Alg. 4 ----------------------------------------------------------------------------

def setup(A, a: float, b: float, params: Params, v0_lanczos: np.ndarray):
    """Set-up of Alg. 4: l1, l2, ||A||, degrees and the coefficients a_j."""
    lmin, lmax, binfo = lanczos_bounds(A, params.lanczos_steps, v0_lanczos, params.bound_pad)
    l1, l2 = cb.linear_map(lmin, lmax)
    normA = max(abs(binfo["theta_min"]), abs(binfo["theta_max"]))
    am, bm = l1 * a + l2, l1 * b + l2
    if not (-1.0 < am < bm < 1.0):
        raise ValueError("interval [a, b] must lie inside the estimated spectrum")
    if params.k_fixed > 0:
        k1 = k = params.k_fixed
    else:
        k1 = cb.initial_degree(am, bm, params.C)
        k = cb.maximum_degree(k1, params.k_ratio)
    coef = cb.filter_coefficients(am, bm, k, params.damping, params.m)
    return dict(lmin=lmin, lmax=lmax, l1=l1, l2=l2, normA=normA, am=am, bm=bm,
                k1=k1, k=k, coef=coef, bounds=binfo)


def adapolysi(A, a: float, b: float, params: Params, V0: np.ndarray,
              v0_lanczos: np.ndarray) -> Result:
    """Alg. 4: FSI with adaptive polynomial filtering.

    A: scipy sparse Hermitian (both triangles).  V0: n x p start block (made
    orthonormal here).  Returns the locked pairs sorted ascending.
    """
    t0 = time.perf_counter()
    S = setup(A, a, b, params, v0_lanczos)
    l1, l2, normA, coef = S["l1"], S["l2"], S["normA"], S["coef"]
    Vhat = cholqr2(np.array(V0, dtype=np.complex128 if np.iscomplexobj(A.data) else np.float64))
    n = A.shape[0]
    Lam = np.zeros(0)
    Vlock = np.zeros((n, 0), dtype=Vhat.dtype)
    n_lock = 0
    n_check_prev = 0
    ki = S["k1"]
    hist = []
    status = "no_convergence"
    spmv_cols = 0
    for it in range(1, params.max_iter + 1):
        # filtering with Alg. 2
        X = clenshaw_apply(A, coef[:ki + 1], l1, l2, Vhat)
        spmv_cols += ki * X.shape[1]
        # orthogonalisation against the locked V, then CholQR2
        X = project_out(Vlock, X)
        Q = cholqr2(X)
        # Rayleigh-Ritz (Alg. 1)
        lam, Vhat = rayleigh_ritz(A, Q)
        spmv_cols += Q.shape[1]
        res = residual_norms(A, Vhat, lam)
        spmv_cols += Q.shape[1]
        # in-interval index set and count
        I = np.nonzero((lam >= a) & (lam <= b))[0]
        e = I.size
        rec = dict(iter=it, degree=ki, width=Vhat.shape[1], e=e, n_lock=n_lock,
                   max_res_in=float(res[I].max() / normA) if e else None)
        if e == 0:                       # nothing inside: next iteration
            hist.append(rec)
            continue
        # next degree by Alg. 3 (fixed-degree runs keep k)
        k_next = cb.degree_select(lam, e, coef, l1, l2, params.tau_a) \
            if params.k_fixed == 0 else ki
        # spurious-eigenvalue test (Eq. (tau_s), Sec. 3.3.2)
        if params.spurious_rule:
            ts = tau_s(lam[I], a, b)
            Cset = I[res[I] < ts]
            n_check = Cset.size + n_lock
            if n_check > 0 and n_check == n_check_prev:
                I = Cset
            n_check_prev = n_check
            rec["tau_s"] = ts
            rec["n_check"] = n_check
        # lock converged pairs (Sec. 3.3.3)
        Lset = I[res[I] <= params.tau_c * normA]
        rec["locked"] = int(Lset.size)
        hist.append(rec)
        done = np.setdiff1d(I, Lset).size == 0
        if params.locking:
            Lam = np.concatenate([Lam, lam[Lset]])
            Vlock = np.concatenate([Vlock, Vhat[:, Lset]], axis=1)
            Vhat = Vhat[:, np.setdiff1d(np.arange(lam.size), Lset)]
            n_lock += Lset.size
        elif done:                       # no deflation: take the pairs at the end
            Lam = lam[I]
            Vlock = Vhat[:, I]
        ki = k_next
        # stop when every in-interval pair is locked
        if done:
            status = "ok"
            break
    order = np.argsort(Lam, kind="stable")
    Lam = Lam[order]
    Vlock = Vlock[:, order]
    rres = residual_norms(A, Vlock, Lam) / normA if Lam.size else np.zeros(0)
    degs = [h["degree"] for h in hist]
    return Result(eigvals=Lam, eigvecs=Vlock, residuals=rres, status=status,
                  stats=dict(setup=S, history=hist, iterations=len(hist),
                             avg_degree=float(np.mean(degs)) if degs else 0.0,
                             spmv_cols=spmv_cols, seconds=time.perf_counter() - t0))
