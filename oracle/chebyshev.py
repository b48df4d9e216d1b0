"""Scalar Chebyshev mathematics of the adaptive filter, in FP64.

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Straight transcriptions of the
definitions in Secs. 2.2 and 3 of the paper; no blocking, fusion or reordering.

Notation: A's spectrum [lmin, lmax] is mapped to [-1, 1] by l(x) = l1 x + l2.
``am``, ``bm`` are the interval ends in mapped coordinates, l(a) and l(b).
alpha = arccos(am), beta = arccos(bm), so alpha > beta.
"""
from __future__ import annotations

import math

import numpy as np

DAMP_LANCZOS_M = "lanczos_m"
DAMP_JACKSON = "jackson"
DAMP_LANCZOS = "lanczos"
DAMP_NONE = "none"


# --- Sec. 2.2: the linear map l(x) ------------------------------------------

def linear_map(lmin: float, lmax: float):
    """l(x) = (2x - lmax - lmin) / (lmax - lmin) = l1 x + l2 (Sec. 2.2)."""
    l1 = 2.0 / (lmax - lmin)
    l2 = -(lmax + lmin) / (lmax - lmin)
    return l1, l2


# --- Eq. (step_func): the step function ------------------------------------------------

def step_function(x, a: float, b: float):
    """s(x): 1 on (a, b), 1/2 at a and b, 0 elsewhere (Eq. (step_func))."""
    x = np.asarray(x, dtype=np.float64)
    out = np.where((x > a) & (x < b), 1.0, 0.0)
    out = np.where((x == a) | (x == b), 0.5, out)
    return out


# --- Eq. (c_j): Chebyshev (Fourier) coefficients of the step function -------------

def step_coefficients(am: float, bm: float, k: int) -> np.ndarray:
    """c_0 .. c_k of s on [-1, 1] for the mapped interval [am, bm] (Eq. (c_j)).

    c_0 = (arccos am - arccos bm) / pi,
    c_j = (2/pi) (sin(j arccos am) - sin(j arccos bm)) / j,   j > 0.
    """
    alpha = math.acos(am)
    beta = math.acos(bm)
    c = np.empty(k + 1, dtype=np.float64)
    c[0] = (alpha - beta) / math.pi
    for j in range(1, k + 1):
        c[j] = (2.0 / math.pi) * (math.sin(j * alpha) - math.sin(j * beta)) / j
    return c


# --- Sec. 2.2 and Eq. (m_Lanczos_damping): damping factors ---------------------------------------

def jackson_damping(k: int) -> np.ndarray:
    """Jackson factors d^J_{j,k}, j = 0..k (Sec. 2.2); the formula gives d_0 = 1."""
    d = np.empty(k + 1, dtype=np.float64)
    t = math.pi / (k + 2)
    for j in range(k + 1):
        d[j] = ((k + 2 - j) * math.sin(t) * math.cos(j * t)
                + math.cos(t) * math.sin(j * t)) / ((k + 2) * math.sin(t))
    return d


def lanczos_m_damping(k: int, m: float) -> np.ndarray:
    """Exponent-m Lanczos factors (sin(j pi/(k+1)) / (j pi/(k+1)))^m (Eq. (m_Lanczos_damping)).

    m = 1 gives the Lanczos sigma factors; d_0 = 1 (the limit of sinc at 0).
    """
    d = np.empty(k + 1, dtype=np.float64)
    d[0] = 1.0
    for j in range(1, k + 1):
        u = j * math.pi / (k + 1)
        d[j] = (math.sin(u) / u) ** m
    return d


def damping(k: int, kind: str = DAMP_LANCZOS_M, m: float = 0.5) -> np.ndarray:
    if kind == DAMP_JACKSON:
        return jackson_damping(k)
    if kind == DAMP_LANCZOS:
        return lanczos_m_damping(k, 1.0)
    if kind == DAMP_LANCZOS_M:
        return lanczos_m_damping(k, m)
    if kind == DAMP_NONE:
        return np.ones(k + 1)
    raise ValueError(kind)


def filter_coefficients(am: float, bm: float, k: int, kind: str = DAMP_LANCZOS_M,
                        m: float = 0.5) -> np.ndarray:
    """a_j = c_j d_{j,k}, j = 0..k: the coefficients of rho^m_{k,k} (Eq. (AdaPolySI)).

    Truncating the returned array at k^(i) <= k gives the adaptive filter of
    Eq. (AdaPolySI), whose damping factors stay those of the maximum degree k.
    """
    return step_coefficients(am, bm, k) * damping(k, kind, m)


# --- Definition of the series, and Alg. 2 on a scalar -----------------------

def cheb_direct(a: np.ndarray, x) -> np.ndarray:
    """sum_j a_j T_j(x) with T_j(x) = cos(j arccos x), for |x| <= 1."""
    x = np.asarray(x, dtype=np.float64)
    th = np.arccos(np.clip(x, -1.0, 1.0))
    out = np.zeros_like(x)
    for j in range(len(a)):
        out = out + a[j] * np.cos(j * th)
    return out


def clenshaw_scalar(a: np.ndarray, l1: float, l2: float, lam) -> np.ndarray:
    """Alg. 2 with A replaced by the scalar(s) lam and X = 1: rho(l(lam)).

    The first step b_{k-1} = 2 l(A) (a_k Y) + a_{k-1} Y is the division-free
    form of the printed line (which divides by a_k and fails when a_k = 0).
    """
    lam = np.asarray(lam, dtype=np.float64)
    k = len(a) - 1
    Y = np.ones_like(lam)
    if k == 0:
        return a[0] * Y
    W = a[k] * Y
    if k == 1:
        return l1 * lam * W + l2 * W + a[0] * Y
    V = 2.0 * l1 * lam * W + 2.0 * l2 * W + a[k - 1] * Y
    V, W = W, V
    for j in range(k - 2, 0, -1):
        V = 2.0 * l1 * lam * W + 2.0 * l2 * W - V + a[j] * Y
        V, W = W, V
    return l1 * lam * W + l2 * W - V + a[0] * Y


# --- Eq. (compute_k_1) and Sec. 4: initial and maximum degree ------------------------------

def initial_degree(am: float, bm: float, C: float = 1.4) -> int:
    """k^(1) = ceil(C / (alpha - beta)) - 1 (Eq. (compute_k_1))."""
    return int(math.ceil(C / (math.acos(am) - math.acos(bm)))) - 1


def maximum_degree(k1: int, ratio: float = 2.5) -> int:
    """k = ceil(2.5 k^(1)) (Sec. 4, parameter settings)."""
    return int(math.ceil(ratio * k1))


# --- Alg. 3: degree for the next iteration -----------------------------------

def degree_select(ritz, e: int, a: np.ndarray, l1: float, l2: float,
                  tau_a: float) -> int:
    """Alg. 3: the smallest j <= k at which the partial filter sum
    gamma_j(x) = sum_{t <= j} a_t T_t(l(x)) over the Ritz values satisfies
    |gamma|_(p) < tau_a |gamma|_(e), where |gamma|_(1) >= ... >= |gamma|_(p) are
    the sorted magnitudes; k (= len(a) - 1) when no j does.

    The T_t(l(x)) come from the three-term recurrence h_next = 2 l(x) h1 - h0.
    The ratio test is written as a product so that a zero |gamma|_(e) does not
    divide.
    """
    ritz = np.asarray(ritz, dtype=np.float64)
    p = ritz.size
    k = len(a) - 1
    if e < 1 or e > p:
        return k
    x = l1 * ritz + l2
    h0 = np.ones(p)
    h1 = x.copy()
    gam = a[0] * h0
    for j in range(1, k + 1):
        gam = gam + a[j] * h1
        s = np.sort(np.abs(gam))[::-1]
        if s[p - 1] < tau_a * s[e - 1]:
            return j
        hn = 2.0 * x * h1 - h0
        h0, h1 = h1, hn
    return k


# --- Sec. 3.2: error bounds ------------------------------------------------------

def S_k(x, k: int):
    """Partial sum sum_{j=1}^k sin(jx)/j of the series of (pi - x)/2 (Lemma 3.1)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for j in range(1, k + 1):
        out = out + np.sin(j * x) / j
    return out


def R_k(x, k: int):
    """R_k(x) = (pi - x)/2 - S_k(x) (Lemma 3.1)."""
    x = np.asarray(x, dtype=np.float64)
    return (math.pi - x) / 2.0 - S_k(x, k)


def lemma31_bound(x, k: int):
    """|R_k(x)| <= 1 / ((k+1) sin(x/2)) for x in (0, pi] (Lemma 3.1)."""
    return 1.0 / ((k + 1) * np.sin(np.asarray(x, dtype=np.float64) / 2.0))


def J_theta(theta, alpha: float, beta: float):
    """J(theta) of Eq. (J_theta) (Thm 3.2), including its values at alpha and beta."""
    th = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    out = np.empty_like(th)
    for i, t in enumerate(th):
        if t == alpha:
            out[i] = (1.0 / abs(math.sin(alpha)) + 1.0 / abs(math.sin((alpha + beta) / 2))
                      + 1.0 / abs(math.sin((alpha - beta) / 2)))
        elif t == beta:
            out[i] = (1.0 / abs(math.sin(beta)) + 1.0 / abs(math.sin((alpha + beta) / 2))
                      + 1.0 / abs(math.sin((alpha - beta) / 2)))
        else:
            out[i] = (1.0 / abs(math.sin((t + alpha) / 2)) + 1.0 / abs(math.sin((t - alpha) / 2))
                      + 1.0 / abs(math.sin((t + beta) / 2)) + 1.0 / abs(math.sin((t - beta) / 2)))
    return out if np.ndim(theta) else out[0]


def g_step(theta, alpha: float, beta: float):
    """g(theta) = s(cos theta): 1 on (beta, alpha), 1/2 at the ends, else 0 (Sec. 3.2)."""
    th = np.asarray(theta, dtype=np.float64)
    out = np.where((th > beta) & (th < alpha), 1.0, 0.0)
    return np.where((th == alpha) | (th == beta), 0.5, out)


def g_damped(theta, c: np.ndarray, d: np.ndarray, ki: int):
    """g^m_{k^(i),k}(theta) = sum_{j=0}^{k^(i)} c_j d_{j,k} cos(j theta) (Eq. (Fourier_series_damping))."""
    th = np.asarray(theta, dtype=np.float64)
    out = np.zeros_like(th)
    for j in range(ki + 1):
        out = out + c[j] * d[j] * np.cos(j * th)
    return out


def thm32_bound(theta, k: int, alpha: float, beta: float):
    """|g - g_k| <= J(theta) / (pi (k+1)) (Thm 3.2, Eq. (gk_bound))."""
    return J_theta(theta, alpha, beta) / (math.pi * (k + 1))


def remark_J_bound(theta, alpha: float, beta: float):
    """J(theta) <= 4 pi / d(theta), d = min |theta +- alpha|, |theta +- beta| (Remark after Thm 3.2)."""
    th = np.asarray(theta, dtype=np.float64)
    d = np.minimum.reduce([np.abs(th + alpha), np.abs(th - alpha),
                           np.abs(th + beta), np.abs(th - beta)])
    return 4.0 * math.pi / d


def C_m(m: float) -> float:
    """C_m = int_0^pi (sin u)^(m-1) (sin u - u cos u) / u^(m+2) du (Eq. (C_m), Thm 3.3).

    Evaluated with adaptive quadrature; for m < 1 the factor (sin u)^(m-1) has
    an integrable singularity at u = pi, handled by the algebraic weight
    (pi - u)^(m-1) of QUADPACK on the last piece.
    """
    from scipy import integrate

    def f(u):
        return (math.sin(u) ** (m - 1)) * (math.sin(u) - u * math.cos(u)) / u ** (m + 2)

    split = 3.0
    head, _ = integrate.quad(f, 0.0, split, limit=400, epsabs=1e-14, epsrel=1e-12)
    if m >= 1.0:
        tail, _ = integrate.quad(f, split, math.pi, limit=400, epsabs=1e-14, epsrel=1e-12)
    else:
        def g(u):  # f(u) / (pi - u)^(m-1), smooth on [split, pi]
            v = math.pi - u                    # sin(u) = sin(v); sin(v)/v -> 1 at v = 0
            s = math.sin(v) / v if v > 0.0 else 1.0
            return (s ** (m - 1)) * (math.sin(u) - u * math.cos(u)) / u ** (m + 2)
        tail, _ = integrate.quad(g, split, math.pi, weight="alg", wvar=(0.0, m - 1.0),
                                 limit=400, epsabs=1e-14, epsrel=1e-12)
    return head + tail


def thm33_bound(theta, ki: int, k: int, m: float, alpha: float, beta: float, Cm=None):
    """Damped pointwise bound of Thm 3.3 (Eq. (damped_fourier_error_bound))."""
    th = np.asarray(theta, dtype=np.float64)
    if Cm is None:
        Cm = C_m(m) if m > 0 else 0.0
    J = J_theta(th, alpha, beta)
    dk = lanczos_m_damping(k, m)[ki]
    return (dk * J / (math.pi * (ki + 1)) + m * Cm * J / (k + 1)
            + m * math.pi * (math.pi - th) / (3.0 * (k + 1) ** 2))


def thm34_bound(Jstar: float, ki: int, k: int, m: float, Cm=None) -> float:
    """Bound on ||P - P^(i)||_2 of Thm 3.4 (Eq. (spectral_proj_error_bound))."""
    if Cm is None:
        Cm = C_m(m) if m > 0 else 0.0
    dk = lanczos_m_damping(k, m)[ki]
    return (dk * Jstar / (math.pi * (ki + 1)) + m * Cm * Jstar / (k + 1)
            + m * math.pi ** 2 / (3.0 * (k + 1) ** 2))
