"""Plain, slow FP64 CPU oracle for adaptive polynomial filtering (AdaPolySI).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it; the seeded input generators in
``synth`` are the only module both sides use.

Modules, each following the paper of Xu, Ni, Li and Zhang, "Adaptive Polynomial
Filtering for Hermitian Interior Eigenproblems":

* ``chebyshev`` -- step-function Chebyshev coefficients (Eq. (c_j)), the linear
  map l(x) (Sec. 2.2), damping factors (Jackson, Lanczos sigma, exponent-m,
  Eq. (m_Lanczos_damping)), scalar Clenshaw (Alg. 2), the initial degree
  (Eq. (compute_k_1)), degree
  selection (Alg. 3) and the error bounds of Lemma 3.1, Thm 3.2, the Remark
  after it, Thm 3.3 and Thm 3.4.
* ``filter`` -- Alg. 2 applied to a sparse Hermitian matrix and a block.
* ``dense`` -- the definition of the result (all eigenpairs in [a, b]) by dense
  eigendecomposition, and an eigenvalue count by Sylvester inertia.
* ``fsi`` -- Lanczos spectrum bounds (Sec. 3.4), Cholesky QR, Rayleigh-Ritz
  (Alg. 1), and the whole of Alg. 4 (AdaPolySI) step by step.
* ``trace`` -- the eigenvalue count estimate (Hutchinson trace of the filter)
  and the subspace size p = ceil(mu e~) of Sec. 3.4.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, quadrature, brute force or the paper's theorems; see
``tests/test_oracle_*.py``.
"""
