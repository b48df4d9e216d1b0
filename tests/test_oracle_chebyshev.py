"""Pins of the oracle's scalar Chebyshev mathematics (no GPU).

Each test checks an oracle function against something other than its own
formula: quadrature, a known kernel property, an identity, or the paper's
theorems evaluated on the oracle's coefficients.
"""
import math

import numpy as np
import pytest

from oracle import chebyshev as cb

INTERVALS = [(-0.3, 0.2), (0.1, 0.6), (-0.95, -0.9), (-0.001, 0.0012), (0.5, 0.99)]


def _gauss(f, lo, hi, n=400):
    x, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
    return 0.5 * (hi - lo) * np.sum(w * f(t))


@pytest.mark.parametrize("am,bm", INTERVALS)
def test_step_coefficients_match_quadrature(am, bm):
    """c_j = (eps_j / pi) int_0^pi s(cos t) cos(j t) dt, eps_0 = 1, eps_j = 2 (Sec. 2.2);
    s(cos t) is the indicator of (beta, alpha), so integrate cos(j t) there."""
    k = 60
    c = cb.step_coefficients(am, bm, k)
    alpha, beta = math.acos(am), math.acos(bm)
    for j in range(k + 1):
        q = _gauss(lambda t: np.cos(j * t), beta, alpha)
        q *= (1.0 if j == 0 else 2.0) / math.pi
        assert abs(c[j] - q) < 1e-13, (j, c[j], q)


@pytest.mark.parametrize("am,bm", INTERVALS[:3])
def test_series_tends_to_step_function(am, bm):
    """The undamped series approaches s(x) (Eq. (step_func)) within Thm 3.2's bound,
    including the value 1/2 at the end points."""
    k = 4000
    c = cb.step_coefficients(am, bm, k)
    alpha, beta = math.acos(am), math.acos(bm)
    xs = np.array([am, bm, 0.5 * (am + bm), am - 0.05, bm + 0.02, -0.999, 0.999])
    xs = xs[(xs > -1) & (xs < 1)]
    val = cb.cheb_direct(c, xs)
    target = cb.step_function(xs, am, bm)
    bound = cb.thm32_bound(np.arccos(xs), k, alpha, beta)
    assert np.all(np.abs(val - target) <= bound + 1e-12)
    assert abs(cb.cheb_direct(c, np.array([am]))[0] - 0.5) < 0.05


@pytest.mark.parametrize("k", [5, 20, 100, 400])
def test_jackson_damped_step_is_positive_and_bounded(k):
    """The Jackson kernel is non-negative with unit mass, so the Jackson-damped
    series of the step function stays in [0, 1] everywhere."""
    am, bm = -0.2, 0.35
    a = cb.step_coefficients(am, bm, k) * cb.jackson_damping(k)
    x = np.cos(np.linspace(0, math.pi, 4001))
    v = cb.cheb_direct(a, x)
    assert v.min() > -1e-13
    assert v.max() < 1.0 + 1e-13


def test_jackson_end_values():
    for k in (1, 7, 50):
        d = cb.jackson_damping(k)
        assert abs(d[0] - 1.0) < 1e-15
        assert np.all(np.diff(d) < 0)
        assert d[-1] > 0


@pytest.mark.parametrize("k", [10, 33, 200])
def test_lanczos_sigma_is_local_average(k):
    """The sigma-damped sum equals the average of the undamped partial sum g_k
    over [theta - h, theta + h], h = pi/(k+1) (the defining property of the
    Lanczos sigma factors)."""
    am, bm = -0.4, 0.1
    c = cb.step_coefficients(am, bm, k)
    d = cb.lanczos_m_damping(k, 1.0)
    h = math.pi / (k + 1)
    for th in (0.3, 1.1, 1.7, 2.9):
        damped = cb.g_damped(np.array([th]), c, d, k)[0]
        avg = _gauss(lambda t: cb.g_damped(t, c, np.ones(k + 1), k), th - h, th + h) / (2 * h)
        assert abs(damped - avg) < 1e-12


def test_lanczos_m_special_cases():
    k = 37
    assert np.allclose(cb.lanczos_m_damping(k, 0.0), 1.0)
    d1 = cb.lanczos_m_damping(k, 1.0)
    assert np.allclose(cb.lanczos_m_damping(k, 2.0), d1 ** 2, rtol=1e-14)
    assert np.allclose(cb.damping(k, cb.DAMP_LANCZOS), d1)
    dm = cb.lanczos_m_damping(k, 0.5)
    assert dm[0] == 1.0 and np.all(np.diff(dm) < 0) and dm[-1] > 0


@pytest.mark.parametrize("k", [0, 1, 2, 3, 17, 250])
def test_clenshaw_scalar_matches_direct_sum(k):
    """Alg. 2 on scalars equals sum a_j cos(j arccos l(lambda))."""
    a = np.cos(np.arange(k + 1) * 1.7) / (1 + np.arange(k + 1))
    lmin, lmax = -3.0, 5.0
    l1, l2 = cb.linear_map(lmin, lmax)
    lam = np.linspace(lmin, lmax, 301)
    v1 = cb.clenshaw_scalar(a, l1, l2, lam)
    v2 = cb.cheb_direct(a, l1 * lam + l2)
    assert np.max(np.abs(v1 - v2)) < 1e-12 * max(1, np.sum(np.abs(a)))


def test_clenshaw_handles_zero_leading_coefficient():
    """Symmetric interval: odd c_j vanish, so a_k = 0 at odd k; Alg. 2's printed
    first step would divide by zero, the division-free form does not."""
    am, bm = -0.3, 0.3
    a = cb.filter_coefficients(am, bm, 41)
    assert abs(a[41]) < 1e-15
    lam = np.linspace(-1, 1, 101)
    v1 = cb.clenshaw_scalar(a, 1.0, 0.0, lam)
    v2 = cb.cheb_direct(a, lam)
    assert np.all(np.isfinite(v1)) and np.max(np.abs(v1 - v2)) < 1e-13


def test_linear_map_endpoints():
    l1, l2 = cb.linear_map(-2.5, 7.0)
    assert abs(l1 * -2.5 + l2 + 1) < 1e-15 and abs(l1 * 7.0 + l2 - 1) < 1e-15


def test_initial_degree_symmetric_interval():
    """For [-b, b]: arccos(-b) - arccos(b) = 2 arcsin(b), so Eq. (compute_k_1)
    reads k1 = ceil(C / (2 arcsin b)) - 1."""
    for b in (0.001, 0.01, 0.2):
        assert cb.initial_degree(-b, b, 1.4) == math.ceil(1.4 / (2 * math.asin(b))) - 1
    assert cb.maximum_degree(97) == 243


def test_degree_select_returns_minimal_degree():
    """Alg. 3 returns the first j where the ratio test holds; checked here by
    direct trigonometric evaluation of the partial sums."""
    am, bm = -0.05, 0.05
    a = cb.filter_coefficients(am, bm, 600)
    ritz = np.concatenate([np.linspace(-0.04, 0.04, 6), np.linspace(0.08, 0.2, 6)])
    e = 6
    j = cb.degree_select(ritz, e, a, 1.0, 0.0, 1e-3)
    assert 1 <= j < 600

    def ok(jj):
        g = np.sort(np.abs(cb.cheb_direct(a[:jj + 1], ritz)))[::-1]
        return g[-1] < 1e-3 * g[e - 1]
    assert ok(j)
    assert not any(ok(jj) for jj in range(1, j))
    # a looser threshold never needs a higher degree
    assert cb.degree_select(ritz, e, a, 1.0, 0.0, 1e-1) <= j
    # e = p: ratio is 1, never below tau_a, so the maximum degree is returned
    assert cb.degree_select(ritz, ritz.size, a, 1.0, 0.0, 1e-3) == 600


# --- Sec. 3.2 theorems, evaluated on the oracle's coefficients -----------------------

@pytest.mark.parametrize("k", [1, 2, 5, 10, 50, 100, 1000])
def test_lemma31(k):
    x = np.linspace(1e-3, math.pi, 2000)
    assert np.all(np.abs(cb.R_k(x, k)) <= cb.lemma31_bound(x, k) * (1 + 1e-12))


def test_Rk_closed_form_limit():
    """R_0 = (pi - x)/2 - 0 and R_k -> 0 pointwise (Lemma 3.1 proof)."""
    x = np.array([0.5, 1.0, 2.0, 3.0])
    assert np.allclose(cb.R_k(x, 0), (math.pi - x) / 2)
    assert np.all(np.abs(cb.R_k(x, 20000)) < 3e-4)


@pytest.mark.parametrize("am,bm", [(0.1, 0.6), (-0.3, 0.2), (-0.9, 0.8)])
@pytest.mark.parametrize("k", [1, 3, 10, 40, 150])
def test_thm32_undamped_bound(am, bm, k):
    alpha, beta = math.acos(am), math.acos(bm)
    c = cb.step_coefficients(am, bm, k)
    th = np.linspace(0, math.pi, 1501)
    th = np.concatenate([th, [alpha, beta]])
    err = np.abs(cb.g_step(th, alpha, beta) - cb.g_damped(th, c, np.ones(k + 1), k))
    assert np.all(err <= cb.thm32_bound(th, k, alpha, beta) * (1 + 1e-12))


def test_remark_J_bound():
    alpha, beta = math.acos(0.1), math.acos(0.6)
    th = np.linspace(0.01, math.pi - 0.01, 999)
    th = th[(np.abs(th - alpha) > 1e-6) & (np.abs(th - beta) > 1e-6)]
    assert np.all(cb.J_theta(th, alpha, beta) <= cb.remark_J_bound(th, alpha, beta) * (1 + 1e-12))


def test_C_m_values():
    """C_m by quadrature against an independent midpoint rule after the
    substitution u = pi - v^2 (which removes the end-point singularity)."""
    for m in (0.5, 1.0, 2.0, 3.0):
        ref_n = 400000
        # piece [0, 3] by midpoint rule, piece [3, pi] by substitution
        u = (np.arange(ref_n) + 0.5) * (3.0 / ref_n)
        f = lambda u: np.sin(u) ** (m - 1) * (np.sin(u) - u * np.cos(u)) / u ** (m + 2)
        head = np.sum(f(u)) * 3.0 / ref_n
        vmax = math.sqrt(math.pi - 3.0)
        v = (np.arange(ref_n) + 0.5) * (vmax / ref_n)
        tail = np.sum(f(math.pi - v * v) * 2 * v) * vmax / ref_n
        assert abs(cb.C_m(m) - (head + tail)) < 1e-6 * (head + tail)
        assert cb.C_m(m) > 0


def test_thm33_fig1_parameters():
    """Thm 3.3 at the parameters of the paper's Fig. 1: a = 0.1, b = 0.6, m = 0.5,
    k = 2.5 k^(i); x = cos(theta) = 0.3 over k^(i); and k = 100 over x in [-0.1, 0.3]."""
    am, bm, m = 0.1, 0.6, 0.5
    alpha, beta = math.acos(am), math.acos(bm)
    Cm = cb.C_m(m)
    th03 = np.array([math.acos(0.3)])
    for ki in (2, 4, 8, 16, 32, 64, 128, 256):
        k = int(math.ceil(2.5 * ki))
        c = cb.step_coefficients(am, bm, k)
        d = cb.lanczos_m_damping(k, m)
        err = abs(cb.g_step(th03, alpha, beta) - cb.g_damped(th03, c, d, ki))[0]
        assert err <= cb.thm33_bound(th03, ki, k, m, alpha, beta, Cm)[0]
    k = 100
    c = cb.step_coefficients(am, bm, k)
    d = cb.lanczos_m_damping(k, m)
    th = np.arccos(np.linspace(-0.1, 0.3, 401))
    for ki in (20, 40, 100):
        err = np.abs(cb.g_step(th, alpha, beta) - cb.g_damped(th, c, d, ki))
        assert np.all(err <= cb.thm33_bound(th, ki, k, m, alpha, beta, Cm))


def test_thm33_reduces_to_thm32_at_m0():
    alpha, beta = math.acos(-0.2), math.acos(0.4)
    th = np.linspace(0.05, 3.0, 50)
    b0 = cb.thm33_bound(th, 30, 75, 0.0, alpha, beta, Cm=0.0)
    assert np.allclose(b0, cb.thm32_bound(th, 30, alpha, beta))


def test_thm34_spectral_projector_bound():
    """||P - P^(i)||_2 <= Eq. (spectral_proj_error_bound) on a small dense
    Hermitian matrix, with P = s(A) and P^(i) = rho(A) formed by eigendecomposition."""
    rs = np.random.default_rng(3)
    n = 60
    M = rs.standard_normal((n, n)) + 1j * rs.standard_normal((n, n))
    A = 0.5 * (M + M.conj().T)
    lam, U = np.linalg.eigh(A)
    lmin, lmax = lam[0] - 0.1, lam[-1] + 0.1
    l1, l2 = cb.linear_map(lmin, lmax)
    a, b = -1.0, 2.5
    am, bm = l1 * a + l2, l1 * b + l2
    m = 0.5
    Cm = cb.C_m(m)
    x = l1 * lam + l2
    Jstar = max(cb.J_theta(np.arccos(x), math.acos(am), math.acos(bm)))
    for ki, k in ((10, 25), (40, 100), (120, 300)):
        coef = cb.filter_coefficients(am, bm, k, cb.DAMP_LANCZOS_M, m)[:ki + 1]
        P = (U * cb.step_function(lam, a, b)) @ U.conj().T
        Pi = (U * cb.cheb_direct(coef, x)) @ U.conj().T
        assert np.linalg.norm(P - Pi, 2) <= cb.thm34_bound(Jstar, ki, k, m, Cm)
