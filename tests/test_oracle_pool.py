"""The column-parallel driver of the oracle's Alg. 2 equals one call of the
oracle on the whole block, bit for bit (no GPU)."""
import numpy as np

from oracle import chebyshev as cb
from oracle import fsi
from oracle.filter import clenshaw_apply
from oracle_pool import clenshaw_apply_parallel
from synth import matrices, rng


def test_parallel_columns_equal_one_call():
    for A in (matrices.anderson(9, 3, 4.0, 3, True), matrices.ks_like_3d(10, 2, n_wells=4)):
        As = A.to_scipy()
        l1, l2 = cb.linear_map(*fsi.gershgorin(As))
        coef = cb.filter_coefficients(-0.2, 0.1, 30)
        X = rng.uniform_block(4, rng.STREAM_TEST, A.n, 13, A.is_complex)
        assert np.array_equal(clenshaw_apply_parallel(A, coef, l1, l2, X, workers=3),
                              clenshaw_apply(As, coef, l1, l2, X))
