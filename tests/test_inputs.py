"""Pins for the seeded input generators (CPU only)."""
import numpy as np
import pytest

import bminputs as bi
from bminputs.philox import philox4x64_10, philox_words


def test_philox_known_answer_vectors():
    # Published known-answer vectors of Philox4x64-10 (Random123 test suite).
    out = philox4x64_10(0, 0, 0, 0, 0, 0)
    assert [int(x) for x in out] == [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC,
                                     0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


@pytest.mark.parametrize("ctr,key", [((10, 3, 0, 9), (5, 7)),
                                     ((2**64 - 2, 2**63, 1, 0), (2**64 - 1, 12345)),
                                     ((0, 0, 0, 0), (0, 0))])
def test_philox_matches_numpy_bit_generator(ctr, key):
    # numpy.random.Philox is Philox4x64-10; it increments the counter before
    # producing its first block of four words.
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(ctr, dtype=np.uint64))
    ref = [int(x) for x in bg.random_raw(4)]
    c0 = (ctr[0] + 1) % 2**64
    c1 = ctr[1] + (1 if c0 == 0 else 0)
    got = [int(x) for x in philox4x64_10(c0, c1, ctr[2], ctr[3], key[0], key[1])]
    assert got == ref


def test_philox_words_layout_vectorised():
    i = np.arange(13, dtype=np.uint64)
    w = philox_words(7, 3, 2, 1, i)
    for q in range(13):
        blk = philox4x64_10(q >> 2, 1, 3, 2, 7, 0)
        assert int(w[q]) == int(blk[q & 3])


def test_mulhi_exact():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2**64, size=200, dtype=np.uint64)
    b = rng.integers(0, 2**64, size=200, dtype=np.uint64)
    hi = bi.u64_mulhi(a, b)
    for x, y, h in zip(a, b, hi):
        assert (int(x) * int(y)) >> 64 == int(h)


def test_unit_double_range_and_exactness():
    w = np.array([0, 2**64 - 1, 2**63], dtype=np.uint64)
    u = bi.u64_to_unit_double(w)
    assert u[0] == 0.0 and u[1] < 1.0 and u[2] == 0.5
    assert u[1] == (2**53 - 1) / 2**53


@pytest.mark.parametrize("m,s", [(20000, 2000), (100, 80), (100, 50), (7, 7),
                                 (1000, 1), (33, 17)])
def test_chunk_indices_are_a_sorted_sample_without_repeats(m, s):
    idx = bi.chunk_indices(0, 3, m, s)
    assert idx.size == s
    assert np.all(np.diff(idx) > 0)
    assert idx.min() >= 0 and idx.max() < m


def test_chunk_indices_uniform():
    # Each row should appear in about s/m of the chunks (chi-square sanity).
    m, s, T = 50, 10, 4000
    cnt = np.zeros(m)
    for t in range(T):
        cnt[bi.chunk_indices(11, t, m, s)] += 1
    expected = T * s / m
    chi2 = ((cnt - expected) ** 2 / expected).sum()
    assert chi2 < 100  # 49 dof: mean 49, p(chi2 > 100) ~ 2e-5


def test_chunk_indices_complement_mode_uniform():
    m, s, T = 20, 15, 4000
    cnt = np.zeros(m)
    for t in range(T):
        cnt[bi.chunk_indices(5, t, m, s)] += 1
    expected = T * s / m
    chi2 = ((cnt - expected) ** 2 / expected).sum()
    assert chi2 < 55   # 19 dof


def test_chunks_differ_and_are_deterministic():
    a = bi.chunk_indices(0, 0, 10000, 500)
    b = bi.chunk_indices(0, 1, 10000, 500)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, bi.chunk_indices(0, 0, 10000, 500))


def test_kpp_uniforms_layout():
    u = bi.kpp_uniforms(4, 9, 5, 3)
    w = philox_words(4, 9, 2, 0, np.arange(15, dtype=np.uint64))
    assert np.array_equal(u.ravel(), bi.u64_to_unit_double(w))
    assert np.all((u >= 0) & (u < 1))


def test_mixture_shapes_and_determinism():
    X = bi.mixtures.blobs_2d()
    assert X.shape == (20000, 2) and X.dtype == np.float32
    assert np.array_equal(X, bi.mixtures.blobs_2d())
    Y, comp = bi.mixtures.anisotropic_with_outliers(5000, 28, 50, 0)
    assert Y.shape == (5000, 28) and (comp == -1).sum() == 50
