"""Random draws that Big-means consumes, laid out on the Philox stream.

Alg. 1 draws a uniform random sample P of s vectors from X for every chunk
(Sec. 3.1, Eq. 2; Sec. 3.5) and K-means++ draws D^2-weighted candidates when
it reseeds degenerate centroids (Sec. 3.3; three candidates per new centre,
Sec. 5).  Both the oracle and the CUDA library consume exactly these numbers:
the oracle receives them from here as inputs, the CUDA library regenerates
them from the same counters with its own Philox.

Purposes (third counter word): 0 = chunk sample, 1 = first K-means++ centre,
2 = K-means++ candidate uniforms.
"""
import numpy as np

from .philox import philox_words, u64_mulhi, u64_to_unit_double

PURPOSE_SAMPLE = 0
PURPOSE_KPP_FIRST = 1
PURPOSE_KPP = 2
MAX_ROUNDS = 64


def _draw_set(seed, t, m, count):
    """The first ``count`` distinct values of the draw sequence in [0, m).

    Round r draws (count - |S|) values v = mulhi(word, m) from counters
    (i, r, t, PURPOSE_SAMPLE), i = 0.., and adds them to S.  Every value that
    enters S is uniform over the values not yet in S, so S is a uniform random
    count-subset.  After MAX_ROUNDS rounds (never reached in practice when
    2*count <= m) the smallest absent values fill the remainder.
    """
    chosen = np.zeros(m, dtype=bool)
    have = 0
    for r in range(MAX_ROUNDS):
        need = count - have
        if need == 0:
            break
        w = philox_words(seed, t, PURPOSE_SAMPLE, r, np.arange(need, dtype=np.uint64))
        v = u64_mulhi(w, np.uint64(m)).astype(np.int64)
        chosen[v] = True
        have = int(chosen.sum())
    if have < count:
        free = np.flatnonzero(~chosen)[: count - have]
        chosen[free] = True
    return chosen


def chunk_indices(seed, t, m, s):
    """Sorted row indices of the sample drawn for chunk ``t`` (size s, no repeats).

    For 2s <= m the sample is the draw set itself; otherwise the m - s rows
    to leave out are drawn and the sample is their complement.
    """
    if not (1 <= s <= m):
        raise ValueError("need 1 <= s <= m")
    if 2 * s <= m:
        chosen = _draw_set(seed, t, m, s)
    else:
        chosen = ~_draw_set(seed, t, m, m - s)
    idx = np.flatnonzero(chosen).astype(np.int64)
    assert idx.size == s
    return idx


def kpp_uniform_first(seed, t):
    """Uniform in [0,1) that picks the first centre when no centroid is live."""
    return float(u64_to_unit_double(philox_words(seed, t, PURPOSE_KPP_FIRST, 0, 0)))


def kpp_uniforms(seed, t, k, trials=3):
    """u[j, l] in [0,1): uniform of candidate l for centroid slot j (k x trials)."""
    i = np.arange(k * trials, dtype=np.uint64)
    w = philox_words(seed, t, PURPOSE_KPP, 0, i)
    return u64_to_unit_double(w).reshape(k, trials)


def chunk_draws(seed, t, m, s, k, trials=3):
    """Everything chunk t consumes: (indices, u_first, u[k, trials])."""
    return (chunk_indices(seed, t, m, s), kpp_uniform_first(seed, t),
            kpp_uniforms(seed, t, k, trials))
