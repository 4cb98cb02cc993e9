"""Counter-based splitmix64 streams (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; the 64-bit finaliser constants are Vigna's published ones).

Draw i (0-based) of the stream with seed S is mix(S + (i + 1) * GOLDEN), where GOLDEN is the
64-bit golden-ratio increment, so any slice of a stream can be produced independently. All
arithmetic is modulo 2**64.

    u   = (draw >> 11) * 2**-53                 in [0, 1)
    U(lo, hi) = lo + (hi - lo) * u
    N(0, 1)   = sqrt(-2 ln(1 - u1)) * cos(2 pi u2)  (Box-Muller on draws 2k, 2k+1)
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def draws(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit draws offset .. offset+n-1 of the stream `seed` (uint64 array)."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (draws(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, n, offset)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller; value k uses draws 2k and 2k+1."""
    u = uniform01(seed, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def integers(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on the closed range [lo, hi]."""
    u = uniform01(seed, n)
    return lo + np.minimum(np.floor(u * (hi - lo + 1)).astype(np.int64), hi - lo)
