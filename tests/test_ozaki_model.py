"""The arithmetic behind the tensor-core Gram product (apf_gram_tc), modelled
on the CPU: columns scaled by their own power of two and cut into seven
signed 8-bit slices, products of slices summed exactly, diagonals s + t <= 6
kept and carried in FP64.  Checked against exact rational arithmetic:

 - each slice is an integer in [-128, 128] (held exactly by bf16) and the
   slices rebuild the value to within 2^(e - 56), exactly when the value is
   within a factor 4 of the column's largest;
 - a 64-row chunk's sums stay below 2^24 (FP32 adds them exactly in any order);
 - the truncated product is within n 2^(e_a + e_b - 53) of the exact one.
"""
from fractions import Fraction

import numpy as np

from synth import rng

S, KC = 7, 64


def _slices(x, e):
    """The device split: t = x 2^-e, then sigma_0 = rint(128 t), sigma_s =
    rint(256 rem) for s >= 1, in FP64."""
    t = np.ldexp(x, -e)
    out = []
    for s in range(S):
        v = t * (128.0 if s == 0 else 256.0)
        sig = np.rint(v)
        t = v - sig
        out.append(sig)
    return np.array(out)  # S x n


def _exponent(col):
    m = np.max(np.abs(col))
    return int(np.frexp(m)[1]) if m > 0 else 0


def test_slices_are_small_integers_and_rebuild_the_value():
    x = rng.uniform_block(3, rng.STREAM_TEST, 500, 1, False)[:, 0] * 7.3
    e = _exponent(x)
    sl = _slices(x, e)
    assert np.all(sl == np.rint(sl)) and np.max(np.abs(sl)) <= 128
    for i in range(0, 500, 7):
        rebuilt = sum(Fraction(int(sl[s, i])) * Fraction(2) ** (e - 7 - 8 * s) for s in range(S))
        err = abs(rebuilt - Fraction(float(x[i])))
        assert err <= Fraction(2) ** (e - 56)
        if abs(x[i]) >= 2.0 ** (e - 2):
            assert err == 0


def test_chunk_sums_fit_fp32_exactly():
    """Worst case: every slice at +-128, seven slice pairs on a diagonal, two
    products per entry (real and imaginary combination), 64 rows."""
    worst = S * 2 * KC * 128 * 128
    assert worst < 2 ** 24


def test_truncated_product_error_bound():
    n, pa, pb = 300, 3, 4
    X = rng.uniform_block(5, rng.STREAM_TEST, n, pa, False) * np.array([1e-3, 1.0, 40.0])
    Y = rng.uniform_block(6, rng.STREAM_TEST, n, pb, False) * np.array([2.0, 1e5, 0.5, 1e-7])
    ex = [_exponent(X[:, a]) for a in range(pa)]
    ey = [_exponent(Y[:, b]) for b in range(pb)]
    SX = [_slices(X[:, a], ex[a]) for a in range(pa)]
    SY = [_slices(Y[:, b], ey[b]) for b in range(pb)]
    for a in range(pa):
        for b in range(pb):
            acc = 0.0
            for c0 in range(0, n, KC):  # chunks: exact integer sums, then the FP64 carry
                for d in range(S):
                    chunk = 0
                    for s in range(d + 1):
                        chunk += int(np.dot(SX[a][s, c0:c0 + KC].astype(np.int64),
                                            SY[b][d - s, c0:c0 + KC].astype(np.int64)))
                    assert abs(chunk) < 2 ** 24
                    acc += float(chunk) * 2.0 ** (-8 * d)
            got = np.ldexp(acc, ex[a] + ey[b] - 14)
            exact = sum(Fraction(float(X[i, a])) * Fraction(float(Y[i, b])) for i in range(n))
            bound = n * Fraction(2) ** (ex[a] + ey[b] - 53)
            assert abs(Fraction(got) - exact) <= bound, (a, b)
