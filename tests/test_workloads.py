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


def test_ks96_interval_agrees_with_the_weyl_count():
    """The stored interval of the 96^3 Kohn-Sham-like workload (from the
    oracle's count estimate) against an independent closed form: away from
    the wells' bound states, -1/2 Laplacian on a periodic box of volume V has
    N(E) ~ V (2E)^(3/2) / (6 pi^2) states below E (Weyl's law for a free
    particle), so [a, b] should hold about N(b) - N(a) eigenvalues.  The wells
    add a few per cent; the estimate said 200."""
    import json
    import os
    w = workloads.ks8_96()
    assert w.p == 300 and 0.0 < w.a < w.b
    vol = 96.0 ** 3
    weyl = lambda E: vol * (2.0 * E) ** 1.5 / (6.0 * np.pi ** 2)  # noqa: E731
    est = weyl(w.b) - weyl(w.a)
    assert 0.8 * 200 <= est <= 1.1 * 200, est
    with open(os.path.join(os.path.dirname(__file__), "golden", "interval_ks8_96.json")) as f:
        d = json.load(f)
    assert abs(d["count_estimate"] - 200.0) < 1.0
    # the bound states of 64 wells of depth 1 sit below zero, a handful per well
    assert 20 <= d["count_below_zero"] <= 64 * 4


def test_c4_slice_workload_shape():
    """Sixteen disjoint contiguous slices, target counts in [20, 150], the
    stored count estimates equal to the targets (the edges were placed by
    them), m = ceil(1.5 count) per slice and more than 1024 columns in all."""
    import json
    import math
    import os
    w = workloads.anderson3d_r_80_slices()
    assert len(w.a) == 16 and w.seed == workloads.BASE_SEED + 3
    with open(os.path.join(os.path.dirname(__file__), "golden", "slices_anderson3d_r_80.json")) as f:
        d = json.load(f)
    assert all(20 <= c <= 150 for c in d["target_counts"])
    assert np.allclose(d["count_estimates"], d["target_counts"], atol=0.5)
    assert w.p == [math.ceil(1.5 * c) for c in d["target_counts"]] and sum(w.p) > 1024
    for s in range(16):
        assert w.a[s] < w.b[s]
        if s:
            assert w.b[s - 1] < w.a[s] and w.a[s] - w.b[s - 1] <= 1e-15
    # the low end of the band: below the clean band edge -6, inside the Gershgorin range -9
    assert -9.0 < w.a[0] and w.b[-1] < -6.0
