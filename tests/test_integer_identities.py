"""The integer identities the sampling kernels rely on for bit-exact draws,
checked exhaustively at the edges and on many random words (no GPU needed):

* Barrett reduction: for 1 <= d < 2^24 and m = floor(2^32 / d) (2^32 - 1 for
  d = 1), q = floor(w m / 2^32) is floor(w / d) or one less, so
  r = w - q d, then r - d if r >= d, is w mod d (the walk step's neighbour
  index and the window split sigma = w mod r);
* division by multiplication (Lemire, Kaser and Kurz): for 32-bit a and
  d >= 2 with M = ceil(2^64 / d), floor(M a / 2^64) = floor(a / d) (the
  tile-local arc of sample s, s / base).
"""
import numpy as np

U32 = (1 << 32) - 1


def barrett_mod(w, d):
    m = U32 if d == 1 else (1 << 32) // d
    q = (w * m) >> 32
    r = w - q * d
    return r - d if r >= d else r


def fastdiv(a, d):
    # the host's magic, floor((2^64 - 1) / d) + 1 = ceil(2^64 / d), fits 64
    # bits for d >= 2 (d = 1 takes s / 1 = s without it)
    assert d >= 2
    M = ((1 << 64) - 1) // d + 1
    assert M < (1 << 64) and M == -(-(1 << 64) // d)
    return (M * a) >> 64


def _words(rng, k):
    edge = [0, 1, 2, 3, U32, U32 - 1, U32 - 2, 1 << 31, (1 << 31) - 1, (1 << 31) + 1]
    return edge + [int(x) for x in rng.integers(0, 1 << 32, k, dtype=np.uint64)]


def test_barrett_reduction_is_exact_for_window_lengths():
    rng = np.random.default_rng(1)
    words = _words(rng, 20000)
    for d in range(1, 17):
        for w in words:
            assert barrett_mod(w, d) == w % d, (w, d)


def test_barrett_reduction_is_exact_for_degrees():
    rng = np.random.default_rng(2)
    degrees = [2, 3, 5, 7, 255, 256, 257, 65535, 65536, 65537, (1 << 24) - 1] + \
        [int(x) for x in rng.integers(2, 1 << 24, 300)]
    for d in degrees:
        words = _words(rng, 200) + [d - 1, d, d + 1, (U32 // d) * d, (U32 // d) * d - 1]
        for w in words:
            w &= U32
            assert barrett_mod(w, d) == w % d, (w, d)


def test_division_by_multiplication_is_exact():
    rng = np.random.default_rng(3)
    divisors = list(range(2, 300)) + [1 << 16, (1 << 16) + 1, 2000, 20000, 667966000] + \
        [int(x) for x in rng.integers(2, 1 << 32, 300, dtype=np.uint64)]
    for d in divisors:
        words = _words(rng, 100) + [d - 1, d, d + 1, (U32 // d) * d, (U32 // d) * d - 1]
        for a in words:
            a &= U32
            assert fastdiv(a, d) == a // d, (a, d)
