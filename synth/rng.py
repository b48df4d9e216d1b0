"""Counter-based SplitMix64 random numbers, keyed by (seed, stream, index).

SplitMix64 is the generator of Steele, Lea and Flood, "Fast splittable
pseudorandom number generators" (OOPSLA 2014): the state advances by the odd
constant GAMMA and each output is the state passed through the 64-bit finaliser
``mix64``.  Used here in counter form: the i-th draw of a stream is the finaliser
applied to ``key(seed, stream) + GAMMA * (i + 1)``, so any draw can be produced
independently of the others (vectorised on the host, one thread per draw on the
device).  The CUDA library carries its own implementation of the same
definition for the initial block and the Lanczos start vector; the two agree bit
for bit.

Uniform doubles take the top 53 bits: ``u = (z >> 11) * 2**-53`` in [0, 1).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids: one per kind of random draw
STREAM_INIT_BLOCK = 1      # initial block V^(0)
STREAM_LANCZOS = 2         # Lanczos start vector for the spectrum bounds
STREAM_TRACE = 3           # probe vectors of the eigenvalue-count estimate
STREAM_POTENTIAL = 10      # on-site disorder / potential values
STREAM_PHASE = 11          # Peierls phases of the bonds
STREAM_CENTRES = 12        # Gaussian well centres
STREAM_TEST = 20           # test blocks


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        return mix64(np.array([s + GAMMA * np.uint64(stream + 1)], dtype=np.uint64))[0]


def raw64(seed: int, stream: int, index) -> np.ndarray:
    """The raw 64-bit draws of one stream at the given indices."""
    key = stream_key(seed, stream)
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + GAMMA * (idx + np.uint64(1)))


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) at the given counter indices."""
    z = raw64(seed, stream, index)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_block(seed: int, stream: int, n: int, p: int, is_complex: bool) -> np.ndarray:
    """An n x p block with entries uniform in [-1, 1), row-major counter order.

    Real entry (i, c) uses counter i*p + c.  Complex entry (i, c) uses counters
    2*(i*p + c) (real part) and 2*(i*p + c) + 1 (imaginary part).
    """
    n = int(n)
    p = int(p)
    if is_complex:
        idx = np.arange(2 * n * p, dtype=np.uint64)
        u = 2.0 * uniform(seed, stream, idx) - 1.0
        return (u[0::2] + 1j * u[1::2]).reshape(n, p)
    idx = np.arange(n * p, dtype=np.uint64)
    return (2.0 * uniform(seed, stream, idx) - 1.0).reshape(n, p)


def rademacher_block(seed: int, stream: int, n: int, m: int) -> np.ndarray:
    """An n x m block of +-1 (real): entry (i, c) is -1 when the uniform draw of
    counter i*m + c is below 1/2, else +1."""
    u = uniform(seed, stream, np.arange(int(n) * int(m), dtype=np.uint64)).reshape(int(n), int(m))
    return np.where(u < 0.5, -1.0, 1.0)
