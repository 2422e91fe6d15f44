"""FP64 CPU oracle of Big-means (Mussabayev, Mladenovic, Mussabayev, Jarboui,
"How to Use K-means for Big Data Clustering?", arXiv 2204.07485).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
reference arm) may import this module.  The CUDA library never calls it and
it shares no code with the CUDA library.

It is the plain, slow, obviously-correct statement of what the GPU path
computes, in float64 (inputs are float32 data promoted to float64).  Random
numbers (chunk indices, K-means++ uniforms) are inputs, drawn by
``bminputs``.  The one library primitive used as a step is
``scipy.spatial.distance.cdist(..., 'sqeuclidean')``, i.e. sum_f (x_f - c_f)^2
evaluated directly in float64.

Readings taken where the paper is silent or ambiguous (each is repeated in the
design notes):
  R1  Eq. 1 is printed without min_j; the text says "nearest centre", so
      f(C, X) = sum_i min_j ||x_i - c_j||^2 over live centroids (Sec. 1).
  R2  Keep-the-best uses Alg. 1 literally: accept C'' iff f(C'', P) < f_opt
      (strict, so a tie keeps the incumbent) (Alg. 1, Sec. 3.2).
  R3  Lloyd stop rule (Sec. 5): stop after an assignment when f == 0, or
      it > 0 and f_prev - f <= tol * f_prev, or it == max_iter (so at most
      max_iter update steps); tol = 1e-4, max_iter = 300.
  R4  f(C'', P) is the objective of the last assignment, computed with the
      returned centroids C'' themselves, so it is exact for C''.
  R5  A centroid that loses all members becomes degenerate (the paper's
      "empty" = "uninitialized" state, Sec. 3.3); it is excluded from later
      assignments of this chunk and reseeded only at the next chunk (Alg. 1).
  R6  Degenerate centroids are excluded from every minimum (treated as +inf).
  R7  K-means++ (Sec. 2, Sec. 3.3, Sec. 5): degenerate slots are filled in
      ascending order on the sample P; if no centroid is live the first one is
      P[floor(u_first * s)]; each further centre draws `trials` (= 3)
      candidates by inverse CDF of D^2 over the inclusive prefix sum in index
      order (smallest i with prefix_i > u * sum D^2; uniform floor(u * s) when
      sum D^2 = 0) and keeps the candidate with the lowest potential
      sum_i min(D^2_i, ||p_i - cand||^2) (lowest trial index on ties).
  R8  The sample is drawn without replacement (indices are an input here).
  R9  Argmin ties go to the lowest centroid index.
  R13 Forgy (Sec. 2: a uniform sample of the data as initial centres) as the
      alternative reinitialisation: each degenerate slot independently takes
      the sample row floor(u * s), u the slot's first K-means++ uniform.
  R12 Parallel modes 2 and 3 (Sec. 3.5): in round r worker w draws chunk
      r * workers + w; "best" means lowest f_opt, lowest worker index on
      ties, and a shared incumbent changes only when strictly improved (as
      R2).  The paper gives no round structure for mode 3; rounds are
      synchronous here.
  R17 Decision following (parity, not the method): a decision whose two
      outcomes are both correct up to FP32 rounding -- an argmin whose top
      two distances differ by less than 1e-5 relative, a stop test or
      keep-the-best comparison within 1e-6 relative of its threshold, a
      K-means++ target within 5e-8 * sum(D^2) of a prefix boundary, or two
      candidate potentials within 1e-6 relative -- is "exempt".  With a
      ``Decisions`` object the run reports every exempt decision it meets
      and takes the other outcome of those named in its ``flips``; the
      arithmetic of every step is unchanged.  A test chooses the flips that
      reproduce the GPU's observed outcome and reports how many it needed.
  R16 The alternative empty-cluster rule ("keep"; the paper names the
      handling of empty clusters as an interchangeable ingredient without
      fixing one): a centroid that loses all members keeps its position and
      stays live, so it can regain members at a later step; R5 is the
      default ("degenerate").
"""
import math

import numpy as np
from scipy.spatial.distance import cdist

# Exemption bands of R17.
TIE_REL = 1e-5          # argmin: (d2 - d1) < TIE_REL * d2
SCALAR_REL = 1e-6       # stop test, keep-the-best, candidate potentials
KPP_BAND = 5e-8         # K-means++ target within KPP_BAND * sum(D^2) of a boundary


class Decisions:
    """Exempt decisions of a run (R17).  ``flips``: keys of the exempt
    decisions that take their other outcome.  ``met`` lists the key of every
    exempt decision the run met, in order.  Keys: ("label", t, it, row),
    ("stop", t, it), ("kpp_target", t, slot, trial), ("kpp_best", t, slot),
    ("keep", t)."""

    def __init__(self, flips=()):
        self.flips = set(flips)
        self.met = []          # (key, relative margin to the decision's threshold)

    def other(self, key, margin):
        """Records an exempt decision; True if it takes the other outcome."""
        self.met.append((key, float(margin)))
        return key in self.flips


# ---------------------------------------------------------------- primitives

def sq_distances(P, C):
    """||p_i - c_j||^2 for all pairs, float64 (s x k).  Sec. 1, Eq. 1."""
    P = np.asarray(P, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    if P.shape[0] == 0 or C.shape[0] == 0:
        return np.zeros((P.shape[0], C.shape[0]))
    return cdist(P, C, "sqeuclidean")


def nearest(P, C, live):
    """Nearest live centroid of every row (R6, R9).

    Returns (labels int64, d1 = squared distance to it, d2 = squared distance
    to the second-nearest live centroid, +inf if only one is live).
    """
    live = np.asarray(live, dtype=bool)
    D = sq_distances(P, C)
    D[:, ~live] = np.inf
    labels = np.argmin(D, axis=1)                 # first minimum: lowest index
    rows = np.arange(D.shape[0])
    d1 = D[rows, labels]
    if live.sum() >= 2:
        D2 = D.copy()
        D2[rows, labels] = np.inf
        d2 = D2.min(axis=1)
    else:
        d2 = np.full(D.shape[0], np.inf)
    return labels, d1, d2


def objective(X, C, live):
    """f(C, X) = sum_i min_{live j} ||x_i - c_j||^2 (Eq. 1 with R1, R6)."""
    _, d1, _ = nearest(X, C, live)
    return float(d1.sum())


# ------------------------------------------------------------ K-means++ (a2)

class KppPick:
    """What one reseeded slot decided, for the tests and the margin report."""

    def __init__(self, slot, cands, potentials, chosen, boundary_margin):
        self.slot = slot
        self.cands = cands
        self.potentials = potentials
        self.chosen = chosen
        self.boundary_margin = boundary_margin


def forgy_reseed(P, C, live, u):
    """Forgy reinitialisation (Sec. 2; R13): every degenerate slot j, in
    ascending order, takes the sample row floor(u[j][0] * s), a uniform pick
    from the sample (independent per slot).  Returns new (C, live) copies."""
    P = np.asarray(P, dtype=np.float64)
    C = np.array(C, dtype=np.float64, copy=True)
    live = np.array(live, dtype=bool, copy=True)
    s = P.shape[0]
    for j in range(C.shape[0]):
        if not live[j]:
            C[j] = P[min(s - 1, int(math.floor(u[j][0] * s)))]
            live[j] = True
    return C, live


def kmeanspp_reseed(P, C, live, u_first, u, trials=3, picks=None, decisions=None, t=0):
    """Reinitialise every degenerate centroid of (C, live) on sample P (R7).

    P: s x n, C: k x n (rows of degenerate slots are ignored), live: k bools,
    u_first: float, u: k x trials uniforms.  Returns new (C, live) copies.
    ``picks`` (optional list) receives one KppPick per reseeded slot.
    ``decisions`` (optional, R17) may take the other outcome of an exempt
    inverse-CDF pick (the neighbouring row with positive D^2 across the
    boundary the target is near) or of an exempt choice between candidates
    (the candidate with the next lowest potential); t names the chunk.
    """
    P = np.asarray(P, dtype=np.float64)
    C = np.array(C, dtype=np.float64, copy=True)
    live = np.array(live, dtype=bool, copy=True)
    s = P.shape[0]
    k = C.shape[0]
    if live.all():
        return C, live
    if not live.any():
        j0 = 0
        C[j0] = P[int(math.floor(u_first * s))]
        live[j0] = True
        D2 = sq_distances(P, C[j0:j0 + 1])[:, 0]
        if picks is not None:
            picks.append(KppPick(j0, [int(math.floor(u_first * s))], [], 0, math.inf))
    else:
        D2 = sq_distances(P, C[live]).min(axis=1)
    for j in range(k):
        if live[j]:
            continue
        total = float(D2.sum())
        prefix = np.cumsum(D2)
        cands, pots, margins = [], [], []
        for l in range(trials):
            if total == 0.0:
                cand = int(math.floor(u[j, l] * s))
                margins.append(math.inf)
            else:
                target = u[j, l] * total
                cand = int(np.searchsorted(prefix, target, side="right"))
                if cand >= s:                       # rounding: last positive D^2
                    cand = int(np.flatnonzero(D2 > 0)[-1])
                lo = prefix[cand - 1] if cand > 0 else 0.0
                below, above = target - lo, prefix[cand] - target
                margins.append(min(below, above) / total)
                if decisions is not None and min(below, above) < KPP_BAND * total:
                    if decisions.other(("kpp_target", t, j, l), min(below, above) / total):
                        pos = np.flatnonzero(D2 > 0)
                        if below <= above:          # the row before the boundary
                            prev = pos[pos < cand]
                            cand = int(prev[-1]) if prev.size else cand
                        else:                       # the row after it
                            nxt = pos[pos > cand]
                            cand = int(nxt[0]) if nxt.size else cand
            dc = sq_distances(P, P[cand:cand + 1])[:, 0]
            cands.append(cand)
            pots.append(float(np.minimum(D2, dc).sum()))
        best = int(np.argmin(pots))                 # lowest trial on ties
        if decisions is not None and trials > 1:
            order = sorted(range(trials), key=lambda q: (pots[q], q))
            b0, b1 = order[0], order[1]
            if pots[b1] - pots[b0] < SCALAR_REL * pots[b0] and cands[b1] != cands[b0]:
                if decisions.other(("kpp_best", t, j), (pots[b1] - pots[b0]) / pots[b0]):
                    best = b1
        C[j] = P[cands[best]]
        live[j] = True
        D2 = np.minimum(D2, sq_distances(P, C[j:j + 1])[:, 0])
        if picks is not None:
            picks.append(KppPick(j, cands, pots, best, min(margins)))
    return C, live


# ------------------------------------------------- Lloyd (a3, a5, a6)

class LloydResult:
    def __init__(self, C, live, f, iters, f_trace, min_gap, stop_margin, n_d):
        self.C = C                  # k x n centroids C''
        self.n_d = n_d              # distance evaluations: s x live per step
        self.live = live            # k bools
        self.f = f                  # f(C'', P), R4
        self.iters = iters          # update steps performed
        self.f_trace = f_trace      # objective of every assignment step
        self.min_gap = min_gap      # min over steps/rows of (d2 - d1) / d2
        self.stop_margin = stop_margin  # min relative distance to the stop threshold


def lloyd(P, C, live, tol=1e-4, max_iter=300, empty="degenerate", decisions=None, t=0):
    """K-means local search on sample P from centroids C (Sec. 2; R3, R4, R5).
    ``empty`` is what happens to a live centroid without members: it becomes
    degenerate (R5) or, with "keep", stays where it is and live (R16).
    ``decisions`` (optional, R17) may give an exempt row its second-nearest
    live centroid or reverse an exempt stop test; t names the chunk."""
    if empty not in ("degenerate", "keep"):
        raise ValueError("empty must be 'degenerate' or 'keep'")
    P = np.asarray(P, dtype=np.float64)
    C = np.array(C, dtype=np.float64, copy=True)
    live = np.array(live, dtype=bool, copy=True)
    k = C.shape[0]
    it = 0
    f_prev = math.inf
    f_trace = []
    min_gap = math.inf
    stop_margin = math.inf
    n_d = 0
    while True:
        n_d += P.shape[0] * int(live.sum())
        labels, d1, d2 = nearest(P, C, live)
        with np.errstate(invalid="ignore", divide="ignore"):
            gaps = np.where(np.isfinite(d2),
                            np.where(d2 > 0, (d2 - d1) / d2, 0.0), np.inf)
        if gaps.size:
            min_gap = min(min_gap, float(np.nanmin(gaps)))
        if decisions is not None:
            for r in np.flatnonzero(gaps < TIE_REL):
                if decisions.other(("label", t, it, int(r)), gaps[r]):
                    dr = sq_distances(P[r:r + 1], C)[0]
                    dr[~live] = np.inf
                    dr[labels[r]] = np.inf
                    labels[r] = int(np.argmin(dr))
                    d1[r] = dr[labels[r]]
        f = float(d1.sum())
        f_trace.append(f)
        stop = f == 0.0 or (it > 0 and f_prev - f <= tol * f_prev) or it == max_iter
        if it > 0 and f_prev > 0:
            margin = abs((f_prev - f) - tol * f_prev) / f_prev
            stop_margin = min(stop_margin, margin)
            if (decisions is not None and margin < SCALAR_REL and f != 0.0
                    and it != max_iter and decisions.other(("stop", t, it), margin)):
                stop = not stop
        if stop:
            break
        for j in range(k):
            if not live[j]:
                continue
            members = P[labels == j]
            if members.shape[0] == 0:
                if empty == "degenerate":
                    live[j] = False
            else:
                C[j] = members.mean(axis=0)
        f_prev = f
        it += 1
    if empty == "degenerate":
        counts = np.bincount(labels, minlength=k)
        live &= counts > 0
    return LloydResult(C, live, f, it, f_trace, min_gap, stop_margin, n_d)


# ------------------------------------------------------- Big-means (Alg. 1)

class ChunkRecord:
    def __init__(self, t, f_chunk, accepted, iters, picks, lloyd_res, keep_margin,
                 n_d):
        self.t = t
        self.n_d = n_d
        self.f_chunk = f_chunk
        self.accepted = accepted
        self.iters = iters
        self.picks = picks
        self.lloyd = lloyd_res
        self.keep_margin = keep_margin


class BigMeansState:
    """Incumbent of Alg. 1: centroids C, live mask, f_opt."""

    def __init__(self, k, n):
        self.C = np.zeros((k, n))
        self.live = np.zeros(k, dtype=bool)
        self.f_opt = math.inf

    def copy(self):
        o = BigMeansState(*self.C.shape)
        o.C = self.C.copy()
        o.live = self.live.copy()
        o.f_opt = self.f_opt
        return o


def big_means_chunk(X, state, idx, u_first, u, tol=1e-4, max_iter=300,
                    trials=3, t=0, init="kmeans++", empty="degenerate", decisions=None):
    """One pass of Alg. 1's loop body on the sample X[idx]; updates ``state``.
    ``init`` chooses the reinitialisation of degenerate centroids: K-means++
    (the paper's choice, R7) or Forgy (R13); ``empty`` the empty-cluster rule
    of Lloyd (R5 or R16); ``decisions`` the exempt decisions of R17."""
    P = np.asarray(X, dtype=np.float32)[np.asarray(idx)].astype(np.float64)
    picks = []
    s = P.shape[0]
    live0 = int(state.live.sum())
    reseeded = state.live.shape[0] - live0
    # n_d of the reseed (Sec. 5 counter): the D^2 of the first centre or of
    # the live set, then `trials` candidate distances per further slot.
    if reseeded == 0 or init == "forgy":
        nd_kpp = 0
    elif live0 == 0:
        nd_kpp = s + (reseeded - 1) * s * trials
    else:
        nd_kpp = s * live0 + reseeded * s * trials
    if init == "forgy":
        C1, live1 = forgy_reseed(P, state.C, state.live, u)
    else:
        C1, live1 = kmeanspp_reseed(P, state.C, state.live, u_first, u, trials, picks,
                                    decisions, t)
    res = lloyd(P, C1, live1, tol, max_iter, empty, decisions, t)
    accepted = res.f < state.f_opt
    keep_margin = (abs(res.f - state.f_opt) / state.f_opt
                   if math.isfinite(state.f_opt) and state.f_opt > 0 else math.inf)
    if (decisions is not None and keep_margin < SCALAR_REL
            and decisions.other(("keep", t), keep_margin)):
        accepted = not accepted
    if accepted:
        state.C = res.C
        state.live = res.live
        state.f_opt = res.f
    return ChunkRecord(t, res.f, accepted, res.iters, picks, res, keep_margin,
                       nd_kpp + res.n_d)


def big_means(X, k, draws, tol=1e-4, max_iter=300, trials=3, state=None,
              t0=0, init="kmeans++", empty="degenerate", decisions=None):
    """Alg. 1 over the given chunk draws [(idx, u_first, u), ...].

    Returns (state, records).  The final assignment is ``final_assignment``.
    """
    X = np.asarray(X, dtype=np.float32)
    if state is None:
        state = BigMeansState(k, X.shape[1])
    records = []
    for q, (idx, u_first, u) in enumerate(draws):
        records.append(big_means_chunk(X, state, idx, u_first, u, tol,
                                       max_iter, trials, t=t0 + q, init=init,
                                       empty=empty, decisions=decisions))
    return state, records


def big_means_workers(X, k, draws_of, workers, rounds, mode, tol=1e-4, max_iter=300,
                      trials=3, state=None, t0=0):
    """The paper's parallel modes (Sec. 3.5), simulated in sequence: in round r
    worker w processes chunk t0 + r * workers + w (draws_of(t) gives its draws).

    mode "competitive" (mode 2): every worker keeps its own incumbent, starting
    from ``state``; after the last round the best worker incumbent (lowest
    f_opt, lowest worker on ties) replaces ``state`` when strictly better.
    mode "collective" (mode 3): every round starts all workers from ``state``;
    the round's best result (same order) replaces ``state`` when strictly
    better.  Returns (state, records of every worker chunk, in (r, w) order).
    """
    X = np.asarray(X, dtype=np.float32)
    if state is None:
        state = BigMeansState(k, X.shape[1])
    mine = [state.copy() for _ in range(workers)]
    records = []
    for r in range(rounds):
        if mode == "collective":
            mine = [state.copy() for _ in range(workers)]
        for w in range(workers):
            t = t0 + r * workers + w
            idx, u_first, u = draws_of(t)
            records.append(big_means_chunk(X, mine[w], idx, u_first, u, tol, max_iter,
                                           trials, t=t))
        if mode == "collective":
            best = min(range(workers), key=lambda w: (mine[w].f_opt, w))
            if mine[best].f_opt < state.f_opt:
                state = mine[best].copy()
    if mode == "competitive":
        best = min(range(workers), key=lambda w: (mine[w].f_opt, w))
        if mine[best].f_opt < state.f_opt:
            state = mine[best].copy()
    return state, records


def final_assignment(X, C, live):
    """Last step of Alg. 1: A_i = nearest live centroid; returns (A, f(C, X))."""
    labels, d1, d2 = nearest(X, C, live)
    return labels, float(d1.sum()), d1, d2
