"""The arithmetic behind the tensor-core products (apf_gram_tc,
apf_block_update with tensor_cores = 1), modelled on the CPU and checked
against exact rational arithmetic:

 - a value x with |x| < 2^E becomes F = round(x 2^(55 - E)), cut into seven
   balanced base-256 digits in [-128, 128] (held exactly by bf16) that rebuild
   F exactly, so x is represented to within 2^(E - 56);
 - a 32-row chunk's digit-product sums on diagonal d stay within
   (d + 1) 2^19, so the kernel's drain period of floor(32 / (d + 1)) chunks
   keeps every FP32 partial sum an integer within 2^24 (exact in any order),
   and the hi / lo carry of the kernel is exact integer arithmetic;
 - the carried sums give the product to within n 2^(E_a + E_b - 55);
 - the digits the model computes equal a direct integer computation from the
   bits of x (the kernel's method) on random, tiny, huge and signed values.
"""
from fractions import Fraction

import numpy as np

from synth import rng

S, KC = 7, 32


def _exponent(v):
    """E with max |v| < 2^E (0 for an all-zero vector)."""
    m = np.max(np.abs(v))
    return int(np.frexp(m)[1]) if m > 0 else 0


def _digits(x, E):
    """Balanced base-256 digits of F = round(x 2^(55 - E)) (halves away from
    zero), low digit last."""
    t = abs(Fraction(float(x))) * Fraction(2) ** (55 - E)
    F = int(t + Fraction(1, 2))  # floor(|t| + 1/2)
    if x < 0:
        F = -F
    dg = [0] * S
    for s in range(S - 1, 0, -1):
        d = F & 0xFF
        if d >= 128:
            d -= 256
        dg[s] = d
        F = (F - d) >> 8
    dg[0] = F
    return dg


def _digits_from_bits(x, E):
    """The kernel's route: mantissa and exponent bits, integer shifts, round
    half away from zero on the magnitude."""
    b = int(np.array([x], dtype=np.float64).view(np.int64)[0])
    ex = (b >> 52) & 0x7FF
    F = 0
    if ex:
        m = (b & ((1 << 52) - 1)) | (1 << 52)
        sh = ex - 1020 - E
        if sh >= 0:
            F = m << min(sh, 2)
        elif sh > -62:
            F = (m + (1 << (-sh - 1))) >> (-sh)
    if b < 0:
        F = -F
    dg = [0] * S
    for s in range(S - 1, 0, -1):
        d = F & 0xFF
        if d >= 128:
            d -= 256
        dg[s] = d
        F = (F - d) >> 8
    dg[0] = F
    return dg


def test_digits_are_small_integers_and_rebuild_the_value():
    x = rng.uniform_block(3, rng.STREAM_TEST, 500, 1, False)[:, 0] * 7.3
    E = _exponent(x)
    for i in range(0, 500, 7):
        dg = _digits(x[i], E)
        assert max(abs(d) for d in dg) <= 128
        rebuilt = sum(Fraction(d) * Fraction(2) ** (E - 55 + 8 * (S - 1 - s)) for s, d in enumerate(dg))
        assert abs(rebuilt - Fraction(float(x[i]))) <= Fraction(2) ** (E - 56)


def test_bit_route_equals_rational_route():
    vals = list(rng.uniform_block(4, rng.STREAM_TEST, 300, 1, False)[:, 0] * 3.0)
    vals += [0.0, -0.0, 1e-300, -1e-300, 2.0 ** -1074, 0.999999999, -0.5, 0.5, 1.5, -1.75]
    # ties: x 2^53 has a fractional part of exactly 1/2 (rounded away from zero)
    vals += [3 * 2.0 ** -54, -5 * 2.0 ** -54, (2 ** 50 + 1) * 2.0 ** -51 + 2.0 ** -54]
    E = 2  # |values| < 4
    for v in vals:
        assert _digits_from_bits(v, E) == _digits(v, E), v
    # the largest magnitude sits right below 2^E
    big = np.nextafter(4.0, 0.0)
    assert _digits_from_bits(big, E) == _digits(big, E)
    assert _digits_from_bits(-big, E) == _digits(-big, E)


def test_chunk_sums_fit_fp32_and_the_carry():
    """Worst case: every digit at +-128, seven digit pairs on a diagonal, 32
    rows: below 2^22.  Carry words: hi gains < 2^36 and lo < 2^46 per chunk, so
    2^16 chunks (the kernel's limit) stay far inside 64 bits."""
    worst = S * KC * 128 * 128
    assert worst < 2 ** 22
    hi = worst * (2 ** 16 + 2 ** 8 + 1)
    lo = worst * (2 ** 24 + 2 ** 16 + 2 ** 8 + 1)
    assert hi * 2 ** 16 < 2 ** 63 and lo * 2 ** 16 < 2 ** 63


def test_drain_periods_keep_fp32_sums_exact():
    """Diagonal d has d + 1 digit pairs: a 32-row chunk adds at most
    (d + 1) x 32 x 128 x 128 = (d + 1) 2^19 to its sum.  The kernel reads the
    FP32 accumulator of d out every floor(32 / (d + 1)) chunks, the longest
    period whose worst case stays within 2^24 (the integers FP32 holds
    exactly); hi and lo then gain less than 2^36 and 2^46 per chunk, so 2^16
    chunks stay inside 64 bits."""
    shift = [16, 8, 0, 24, 16, 8, 0]
    hi = lo = 0
    for d in range(S):
        per = 32 // (d + 1)
        worst = (d + 1) * KC * 128 * 128
        assert per * worst <= 2 ** 24 < (per + 1) * worst
        if d < 3:
            hi += worst << shift[d]
        else:
            lo += worst << shift[d]
    assert hi < 2 ** 36 and lo < 2 ** 46
    assert hi * 2 ** 16 < 2 ** 63 and lo * 2 ** 16 < 2 ** 63


def test_carried_product_error_bound():
    n, pa, pb = 300, 3, 4
    X = rng.uniform_block(5, rng.STREAM_TEST, n, pa, False) * np.array([1e-3, 1.0, 40.0])
    Y = rng.uniform_block(6, rng.STREAM_TEST, n, pb, False) * np.array([2.0, 1e5, 0.5, 1e-7])
    ex = [_exponent(X[:, a]) for a in range(pa)]
    ey = [_exponent(Y[:, b]) for b in range(pb)]
    DX = [[_digits(X[i, a], ex[a]) for i in range(n)] for a in range(pa)]
    DY = [[_digits(Y[i, b], ey[b]) for i in range(n)] for b in range(pb)]
    for a in range(pa):
        for b in range(pb):
            # the kernel's schedule: per-diagonal sums over drain periods of
            # floor(32 / (d + 1)) chunks, carried into hi / lo at each period's end
            hi = lo = 0
            acc = [0] * S
            nch = (n + KC - 1) // KC
            for c in range(nch):
                c0 = c * KC
                for d in range(S):
                    for s in range(d + 1):
                        acc[d] += sum(DX[a][i][s] * DY[b][i][d - s] for i in range(c0, min(n, c0 + KC)))
                    assert abs(acc[d]) <= 2 ** 24
                    if (c + 1) % (32 // (d + 1)) == 0 or c == nch - 1:
                        if d < 3:
                            hi += acc[d] << (16, 8, 0)[d]
                        else:
                            lo += acc[d] << (24, 16, 8, 0)[d - 3]
                        acc[d] = 0
            got = Fraction(hi * 2 ** 32 + lo) * Fraction(2) ** (ex[a] + ey[b] - 62)
            exact = sum(Fraction(float(X[i, a])) * Fraction(float(Y[i, b])) for i in range(n))
            bound = n * Fraction(2) ** (ex[a] + ey[b] - 55)
            assert abs(got - exact) <= bound, (a, b)
