"""Pins of the oracle's matrix-level functions (no GPU): Alg. 2 on matrices,
the dense definition, inertia counts, Lanczos bounds, CholQR2 and Alg. 4."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import chebyshev as cb
from oracle import dense, fsi
from oracle.filter import clenshaw_apply, filter_dense_definition
from synth import matrices, rng, workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_hermitian(n, seed, is_complex):
    A = matrices.random_sparse_hermitian(n, 5, seed, is_complex)
    return A.to_scipy(), A.to_dense()


@pytest.mark.parametrize("is_complex", [False, True])
@pytest.mark.parametrize("k", [0, 1, 2, 7, 60])
def test_clenshaw_matrix_matches_spectral_definition(is_complex, k):
    As, Ad = _small_hermitian(80, 4, is_complex)
    lam = np.linalg.eigvalsh(Ad)
    l1, l2 = cb.linear_map(lam[0] - 0.01, lam[-1] + 0.01)
    a = cb.filter_coefficients(l1 * -0.3 + l2, l1 * 0.4 + l2, max(k, 1))[:k + 1]
    X = rng.uniform_block(9, rng.STREAM_TEST, 80, 7, is_complex)
    V1 = clenshaw_apply(As, a, l1, l2, X)
    V2 = filter_dense_definition(Ad, a, l1, l2, X)
    assert np.max(np.abs(V1 - V2)) < 1e-12 * np.max(np.abs(X)) * max(1.0, np.sum(np.abs(a)))


def test_clenshaw_on_diagonal_is_scalar_series():
    d = np.linspace(-1.9, 2.9, 50)
    A = sp.diags(d).tocsr()
    l1, l2 = cb.linear_map(-2.0, 3.0)
    a = cb.filter_coefficients(l1 * 0.1 + l2, l1 * 0.7 + l2, 33)
    V = clenshaw_apply(A, a, l1, l2, np.eye(50))
    assert np.allclose(np.diag(V), cb.cheb_direct(a, l1 * d + l2), atol=1e-13)
    assert np.allclose(V - np.diag(np.diag(V)), 0.0)


def test_analytic_spectrum_laplacian2d():
    """Zero potential: eigenvalues 4 - 2 cos(pi i/(L+1)) - 2 cos(pi j/(L+1))."""
    L = 12
    A = matrices.laplacian2d_dirichlet(L, 1, pot_halfwidth=0.0)
    i = np.arange(1, L + 1)
    ref = np.sort((4 - 2 * np.cos(np.pi * i[:, None] / (L + 1))
                   - 2 * np.cos(np.pi * i[None, :] / (L + 1))).ravel())
    assert np.allclose(dense.all_eigenvalues(A.to_dense()), ref, atol=1e-12)


def test_analytic_spectrum_anderson3d_clean():
    """W = 0, no phases: eigenvalues -2 (cos 2pi i/L + cos 2pi j/L + cos 2pi k/L)."""
    L = 6
    A = matrices.anderson(L, 3, 0.0, 1, complex_phases=False)
    q = 2 * np.pi * np.arange(L) / L
    ref = np.sort((-2 * (np.cos(q)[:, None, None] + np.cos(q)[None, :, None]
                         + np.cos(q)[None, None, :])).ravel())
    assert np.allclose(dense.all_eigenvalues(A.to_dense()), ref, atol=1e-12)


def test_matrices_are_hermitian():
    for A in (matrices.anderson(5, 3, 4.0, 3, True), matrices.laplacian2d_dirichlet(7, 2),
              matrices.ks_like_3d(9, 2, n_wells=3), matrices.random_sparse_hermitian(50, 4, 1, True)):
        M = A.to_scipy()
        assert abs(M - M.getH()).max() < 1e-15
        assert np.all(np.diff(A.rowptr) > 0)


@pytest.mark.parametrize("is_complex", [False, True])
def test_inertia_count_matches_eigh(is_complex):
    A = matrices.anderson(7, 3, 4.0, 5, is_complex).to_dense()
    lam = np.linalg.eigvalsh(A)
    for s in (-3.1, -0.2, 0.0137, 2.5):
        assert dense.inertia_count_below(A, s) == int(np.sum(lam < s))


def test_golden_interval_lap2d():
    """The stored interval holds the stored eigenvalues; inertia agrees."""
    w = workloads.lap2d_32()
    with open(os.path.join(GOLDEN, "interval_lap2d_32.json")) as f:
        g = json.load(f)
    Ad = w.matrix().to_dense()
    assert dense.interval_count(Ad, w.a, w.b) == g["count"]
    lam, _ = dense.interior_eigenpairs(Ad, w.a, w.b)
    assert np.allclose(lam, g["eigenvalues"], atol=1e-12)


def test_lanczos_bounds_enclose_spectrum():
    for A in (workloads.lap2d_32().matrix(), matrices.anderson(10, 3, 4.0, 7, True),
              matrices.ks_like_3d(10, 1, n_wells=4)):
        As = A.to_scipy()
        lam = np.linalg.eigvalsh(A.to_dense())
        v0 = rng.uniform_block(1, rng.STREAM_LANCZOS, A.n, 1, A.is_complex)[:, 0]
        lmin, lmax, info = fsi.lanczos_bounds(As, 40, v0)
        assert lmin <= lam[0] and lmax >= lam[-1]
        assert lmax - lmin <= 1.05 * (lam[-1] - lam[0])
        g = fsi.gershgorin(As)
        assert g[0] <= lam[0] and g[1] >= lam[-1]


def test_lanczos_tiny_matrix_breakdown():
    """n < steps: the Krylov space is exhausted; the Ritz values are exact."""
    A = sp.diags([1.0, 2.0, 5.0]).tocsr()
    lmin, lmax, info = fsi.lanczos_bounds(A, 40, np.ones(3))
    assert info["steps"] <= 3
    assert abs(info["theta_min"] - 1.0) < 1e-12 and abs(info["theta_max"] - 5.0) < 1e-12


@pytest.mark.parametrize("kappa", [1e3, 1e7, 1e12])
def test_cholqr2(kappa):
    n, p = 500, 12
    G = rng.uniform_block(3, rng.STREAM_TEST, n, p, True)
    Q0, _ = np.linalg.qr(G)
    W = rng.uniform_block(4, rng.STREAM_TEST, p, p, True)
    U, _ = np.linalg.qr(W)
    X = Q0 @ np.diag(np.logspace(0, -math.log10(kappa), p)) @ U
    Q = fsi.cholqr2(X)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(p))) < 1e-13
    # same column space: projecting X onto Q leaves nothing relative to the
    # smallest singular direction's accuracy
    assert np.linalg.norm(X - Q @ (Q.conj().T @ X)) < 1e-10 * np.linalg.norm(X)


def _interval_around(lam, centre, cnt):
    i0 = int(np.searchsorted(lam, centre))
    lo, hi = i0 - cnt // 2, i0 - cnt // 2 + cnt
    return 0.5 * (lam[lo - 1] + lam[lo]), 0.5 * (lam[hi - 1] + lam[hi])


def _check_result(r, As, lam_ref, normA_tol=1e-10):
    assert r.status == "ok"
    assert r.eigvals.size == lam_ref.size
    lam_all = np.abs(np.linalg.eigvalsh(As.toarray())).max()
    assert np.max(np.abs(r.eigvals - lam_ref)) <= 1e-10 * lam_all
    # the lock threshold's ||A|| never exceeds the spectral radius, so the
    # residuals meet the Sec. 4 test against the true ||A||
    normA = r.stats["setup"]["normA"]
    assert 0.5 * lam_all <= normA <= lam_all * (1 + 1e-12)
    V = r.eigvecs
    res = np.linalg.norm(As @ V - V * r.eigvals, axis=0) / lam_all
    assert np.all(res <= normA_tol)
    assert np.max(np.abs(V.conj().T @ V - np.eye(V.shape[1]))) < 1e-10


@pytest.mark.slow
def test_adapolysi_lap2d_workload():
    """Alg. 4 on the 32 x 32 Laplacian workload finds exactly the dense set."""
    w = workloads.lap2d_32()
    A = w.matrix()
    As = A.to_scipy()
    lam_ref, _ = dense.interior_eigenpairs(A.to_dense(), w.a, w.b)
    V0 = rng.uniform_block(w.seed, rng.STREAM_INIT_BLOCK, A.n, w.p, False)
    v0 = rng.uniform_block(w.seed, rng.STREAM_LANCZOS, A.n, 1, False)[:, 0]
    r = fsi.adapolysi(As, w.a, w.b, fsi.Params(p=w.p), V0, v0)
    _check_result(r, As, lam_ref)
    assert r.stats["setup"]["k1"] == cb.initial_degree(r.stats["setup"]["am"], r.stats["setup"]["bm"])


def test_adapolysi_complex_anderson_small():
    A = matrices.anderson(10, 3, 4.0, 7, True)
    As = A.to_scipy()
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _interval_around(lam, 0.0, 11)
    V0 = rng.uniform_block(7, rng.STREAM_INIT_BLOCK, A.n, 20, True)
    v0 = rng.uniform_block(7, rng.STREAM_LANCZOS, A.n, 1, True)[:, 0]
    r = fsi.adapolysi(As, a, b, fsi.Params(p=20), V0, v0)
    _check_result(r, As, lam[(lam >= a) & (lam <= b)])
    assert dense.interval_count(A.to_dense(), a, b) == r.eigvals.size


def _symmetric_stall_matrix(seed):
    cs = np.linspace(0.3, 1.0, 100)
    lam = np.sort(np.concatenate([-cs, cs, [-0.05, -0.02, 0.03, 0.06]]))
    n = lam.size
    Q, _ = np.linalg.qr(rng.uniform_block(seed, rng.STREAM_TEST, n, n, False))
    Ad = (Q * lam) @ Q.T
    return sp.csr_matrix(0.5 * (Ad + Ad.T)), n


def test_spurious_rule_ends_stall():
    """Sec. 3.3.2: with a symmetric spectrum and a symmetric interval the filter
    is even, so a Ritz vector mixing the eigenvectors of +c and -c never
    converges and its Ritz value can sit inside [a, b] with a large residual.
    The tau_s rule removes it and the run ends with exactly the 4 eigenvalues
    inside; without the rule the run reaches the iteration cap."""
    As, n = _symmetric_stall_matrix(2)
    V0 = rng.uniform_block(2, rng.STREAM_INIT_BLOCK, n, 15, False)
    v0 = rng.uniform_block(2, rng.STREAM_LANCZOS, n, 1, False)[:, 0]
    P = dict(p=15, k_fixed=20, damping=cb.DAMP_JACKSON, max_iter=30)
    r = fsi.adapolysi(As, -0.1, 0.1, fsi.Params(**P, spurious_rule=True), V0, v0)
    assert r.status == "ok" and r.stats["iterations"] <= 12
    assert np.allclose(r.eigvals, [-0.05, -0.02, 0.03, 0.06], atol=1e-11)
    assert any(h["e"] > 4 for h in r.stats["history"])   # a spurious value was present
    r2 = fsi.adapolysi(As, -0.1, 0.1, fsi.Params(**P, spurious_rule=False), V0, v0)
    assert r2.status == "no_convergence" and r2.stats["iterations"] == 30


def test_shifted_cholqr_branch_runs_with_the_published_shift(monkeypatch):
    """At kappa = 1e12 the Gram matrix's Cholesky factorisation breaks down
    (kappa^2 > 1/u), so CholQR2 must take the shifted first pass of Fukaya et
    al. (2020).  The shift is 11 (n p + p (p + 1)) u ||X||_F^2: R^H R - X^H X
    equals s I up to rounding, so a shift ten times too large (or too small)
    fails here."""
    n, p = 500, 12
    G = rng.uniform_block(3, rng.STREAM_TEST, n, p, True)
    Q0, _ = np.linalg.qr(G)
    U, _ = np.linalg.qr(rng.uniform_block(4, rng.STREAM_TEST, p, p, True))
    # singular values down to 1e-12, with the last one exactly zero in the
    # Gram matrix's precision: plain Cholesky cannot succeed
    X = Q0 @ np.diag(np.concatenate([np.logspace(0, -12, p - 1), [1e-17]])) @ U
    with pytest.raises(np.linalg.LinAlgError):
        fsi.cholqr(X)
    calls = []
    orig = fsi.shifted_cholqr
    monkeypatch.setattr(fsi, "shifted_cholqr", lambda Z: calls.append(1) or orig(Z))
    Q = fsi.cholqr2(X)
    assert calls == [1]
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(p))) < 1e-12
    _, R = orig(X)
    u = np.finfo(np.float64).eps / 2
    s = 11.0 * (n * p + p * (p + 1)) * u * np.linalg.norm(X) ** 2
    D = R.conj().T @ R - X.conj().T @ X
    assert np.max(np.abs(D - s * np.eye(p))) <= 0.05 * s
    assert np.allclose(np.real(np.diag(D)), s, rtol=0.05)


@pytest.mark.parametrize("is_complex", [False, True])
def test_project_out_is_the_orthogonal_projector(is_complex):
    """X - V (V^H X) twice: the result is orthogonal to the locked V, what was
    removed lies in span(V), projecting again changes nothing, and a block
    already orthogonal to V comes back unchanged (to rounding)."""
    n, m, p = 200, 7, 5
    V, _ = np.linalg.qr(rng.uniform_block(21, rng.STREAM_TEST, n, m, is_complex))
    X = rng.uniform_block(22, rng.STREAM_TEST, n, p, is_complex)
    Y = fsi.project_out(V, X)
    assert np.max(np.abs(V.conj().T @ Y)) < 1e-14 * np.abs(X).max() * n
    D = X - Y                                   # the removed part
    assert np.max(np.abs(D - V @ (V.conj().T @ D))) < 1e-13 * np.abs(X).max()
    assert np.max(np.abs(fsi.project_out(V, Y) - Y)) < 1e-14 * np.abs(X).max() * n
    Z = Y / np.abs(Y).max()
    assert np.max(np.abs(fsi.project_out(V, Z) - Z)) < 1e-13
    assert fsi.project_out(V[:, :0], X) is X   # nothing locked: nothing to remove


@pytest.mark.parametrize("is_complex", [False, True])
def test_rayleigh_ritz_on_an_invariant_subspace(is_complex):
    """Alg. 1 on a basis Q of an invariant subspace (any orthonormal mixing of
    eigenvectors of A) returns exactly those eigenvalues, with Ritz vectors
    that are eigenvectors; on a generic subspace the Ritz values lie inside the
    spectrum and the Ritz vectors are orthonormal."""
    As, Ad = _small_hermitian(90, 8, is_complex)
    lam, U = np.linalg.eigh(Ad)
    idx = [3, 17, 40, 41, 77]
    W, _ = np.linalg.qr(rng.uniform_block(23, rng.STREAM_TEST, len(idx), len(idx), is_complex))
    Q = U[:, idx] @ W                           # same span, mixed basis
    th, V = fsi.rayleigh_ritz(As, Q)
    assert np.max(np.abs(th - lam[idx])) < 1e-12 * np.abs(lam).max()
    assert np.max(fsi.residual_norms(As, V, th)) < 1e-12 * np.abs(lam).max()
    Qg, _ = np.linalg.qr(rng.uniform_block(24, rng.STREAM_TEST, 90, 6, is_complex))
    th, V = fsi.rayleigh_ritz(As, Qg)
    assert np.all(th >= lam[0] - 1e-12) and np.all(th <= lam[-1] + 1e-12)
    assert np.max(np.abs(V.conj().T @ V - np.eye(6))) < 1e-13


def test_residual_norms_of_exact_and_shifted_pairs():
    """||A v - mu v|| is zero (to rounding) for an eigenpair and equals
    |lambda - mu| for an eigenvector of unit norm paired with a wrong value."""
    As, Ad = _small_hermitian(60, 9, True)
    lam, U = np.linalg.eigh(Ad)
    r = fsi.residual_norms(As, U[:, :4], lam[:4])
    assert np.max(r) < 1e-13 * np.abs(lam).max()
    shift = np.array([0.5, -0.25, 1e-3, 2.0])
    r = fsi.residual_norms(As, U[:, :4], lam[:4] + shift)
    assert np.allclose(r, np.abs(shift), rtol=1e-10, atol=1e-13)
