"""Invariants of the seeded workloads the benches and GPU tests use (no GPU):
the serving request stream, the spectrum-slice workload and the stored
interval of the 2D workload."""
import numpy as np

from synth import matrices, workloads


def test_serving_requests_are_seeded_and_in_range():
    a = workloads.serving_requests(24)
    b = workloads.serving_requests(24)
    assert [(r.dim, r.L, r.W, r.is_complex, r.seed, r.a, r.b) for r in a] == \
           [(r.dim, r.L, r.W, r.is_complex, r.seed, r.a, r.b) for r in b]
    dims = {r.dim for r in a}
    assert dims == {2, 3} and {r.is_complex for r in a} == {False, True}
    for r in a:
        n = r.L ** r.dim
        assert 0.5e4 <= n <= 1.2e5
        assert 1.0 <= r.W <= 6.0 and 8 <= r.target <= 64
        half_band = 2.0 * r.dim + r.W / 2.0  # Gershgorin half-width of the model
        assert -half_band / 2 <= r.a < r.b <= half_band / 2
    # the matrix of one request is Hermitian with the model's Gershgorin range
    A = a[0].matrix()
    M = A.to_scipy()
    assert abs(M - M.conj().T).max() == 0.0
    assert np.abs(M).sum(axis=1).max() <= 2.0 * a[0].dim + a[0].W / 2.0 + 1e-12


def test_slice_workload_is_disjoint_and_contiguous():
    w = workloads.anderson3d_r_48_slices()
    assert len(w.a) == len(w.b) == len(w.p) == 8 and all(p == 0 for p in w.p)
    for s in range(8):
        assert w.a[s] < w.b[s]
        if s:
            assert w.b[s - 1] < w.a[s]                    # disjoint
            assert w.a[s] - w.b[s - 1] <= 1e-15           # contiguous up to one ulp
    widths = np.array(w.b) - np.array(w.a)
    assert np.allclose(widths, widths[0], rtol=1e-9)
    assert abs(0.5 * (w.a[0] + w.b[-1])) < 1e-12        # centred on E = 0


def test_lap2d_interval_holds_its_stored_eigenvalues():
    w = workloads.lap2d_32()
    A = matrices.laplacian2d_dirichlet(32, w.seed, 0.5)
    lam = np.linalg.eigvalsh(A.to_dense())
    inside = lam[(lam >= w.a) & (lam <= w.b)]
    assert inside.size == 18
