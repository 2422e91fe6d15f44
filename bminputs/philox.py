"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), vectorised in numpy.

The same generator is written independently in the CUDA library; both follow
the published definition: 10 rounds of two 64x64->128 multiplies with the
constants M0, M1 and a Weyl key schedule W0, W1.  The known-answer vectors of
the published test suite and numpy's own ``numpy.random.Philox`` (which is
Philox4x64-10) pin this implementation in ``tests/test_inputs.py``.

Stream layout used by Big-means (both sides):
  key     = (seed, 0)
  counter = (i >> 2, round, chunk t, purpose);   word = i & 3
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def u64_mulhi(a, b):
    """High 64 bits of the 128-bit product of two uint64 arrays (exact)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    with np.errstate(over="ignore"):
        ll = a_lo * b_lo
        lh = a_lo * b_hi
        hl = a_hi * b_lo
        hh = a_hi * b_hi
        mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
        return hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)


def _mullo(a, b):
    with np.errstate(over="ignore"):
        return np.asarray(a, dtype=np.uint64) * np.asarray(b, dtype=np.uint64)


def philox4x64_10(c0, c1, c2, c3, k0, k1):
    """Return the four 64-bit output words for counters (c0..c3), key (k0, k1).

    Arguments broadcast as uint64 arrays.
    """
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64)
    k1 = np.asarray(k1, dtype=np.uint64)
    for r in range(10):
        hi0, lo0 = u64_mulhi(M0, x0), _mullo(M0, x0)
        hi1, lo1 = u64_mulhi(M1, x2), _mullo(M1, x2)
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        if r != 9:
            with np.errstate(over="ignore"):
                k0 = k0 + W0
                k1 = k1 + W1
    return x0, x1, x2, x3


def philox_words(seed, t, purpose, rnd, i):
    """64-bit draw number ``i`` (array) of stream (seed, chunk t, purpose, round)."""
    i = np.asarray(i, dtype=np.uint64)
    words = philox4x64_10(i >> np.uint64(2), np.uint64(rnd), np.uint64(t),
                          np.uint64(purpose), np.uint64(seed), np.uint64(0))
    sel = (i & np.uint64(3)).astype(np.int64)
    out = np.choose(sel, words) if i.ndim else words[int(sel)]
    return np.asarray(out, dtype=np.uint64)


def u64_to_unit_double(w):
    """Map 64 random bits to a double in [0, 1): top 53 bits times 2^-53 (exact)."""
    w = np.asarray(w, dtype=np.uint64)
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
