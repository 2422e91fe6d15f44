"""Decision following for whole-run parity (the oracle's reading R17).

A free-running GPU run meets decisions whose two outcomes are both correct up
to FP32 rounding (exempt decisions: near-tied rows, a stop test or
keep-the-best comparison at its threshold, a K-means++ target at a prefix
boundary, near-equal candidate potentials).  After each chunk the GPU's
observable outcome -- accepted or not, its Lloyd update steps, and when
accepted the incumbent's mask, objective and centroids -- is compared with
the oracle's.  If they disagree, the oracle's chunk is re-run from the same
state with exempt decisions taking their other outcome (the smallest margins
first, single flips, then pairs) until one reproduces the GPU's outcome; the
flips used are the followed decisions.  Every value compared is computed by
the oracle; the GPU only selects among outcomes the oracle itself admits.
"""
import math

import numpy as np

import oracle as o

OBJ_REL = 1e-6
CEN_REL = 1e-6


def chunk_matches(state_after, rec, obs):
    """obs: dict(accepted, iters, f_opt, C, live) of the GPU after the chunk."""
    if bool(obs["accepted"]) != bool(rec.accepted) or int(obs["iters"]) != int(rec.iters):
        return False
    if not np.array_equal(np.asarray(obs["live"], bool), state_after.live):
        return False
    if math.isfinite(state_after.f_opt):
        if abs(obs["f_opt"] - state_after.f_opt) > OBJ_REL * abs(state_after.f_opt):
            return False
    live = state_after.live
    if live.any():
        err = np.linalg.norm(np.asarray(obs["C"], np.float64)[live] - state_after.C[live], axis=1)
        scale = np.maximum(np.linalg.norm(state_after.C[live], axis=1), 1.0)
        if float((err / scale).max()) > CEN_REL:
            return False
    return True


def follow_chunk(X, state, draw, t, obs, max_flips=2, budget=64, **kw):
    """Runs the oracle's chunk t from `state` (not modified); returns
    (state after, record, flips) for the first flip set whose outcome matches
    `obs`, or None if none within `budget` runs does."""
    idx, uf, u = draw
    queue, seen, tried = [()], {()}, 0
    while queue and tried < budget:
        flips = queue.pop(0)
        st = state.copy()
        d = o.Decisions(flips)
        rec = o.big_means_chunk(X, st, idx, uf, u, t=t, decisions=d, **kw)
        tried += 1
        if chunk_matches(st, rec, obs):
            return st, rec, flips
        if len(flips) < max_flips:
            met = sorted(d.met, key=lambda km: km[1])
            for key, _ in met:
                if key in flips:
                    continue
                nf = tuple(sorted(flips + (key,), key=repr))
                if nf not in seen:
                    seen.add(nf)
                    queue.append(nf)
    return None


def follow_run(X, k, draws, observe, t0=0, **kw):
    """Follows a whole run chunk by chunk.  observe(t) runs the GPU's chunk t
    and returns its outcome (see chunk_matches).  Returns (state, records,
    followed flips, first failing chunk or None)."""
    state = o.BigMeansState(k, np.asarray(X).shape[1])
    recs, followed = [], []
    for q, draw in enumerate(draws):
        t = t0 + q
        obs = observe(t)
        hit = follow_chunk(X, state, draw, t, obs, **kw)
        if hit is None:
            return state, recs, followed, t
        state, rec, flips = hit
        recs.append(rec)
        followed.extend(flips)
    return state, recs, followed, None


def _assign_block(args):
    """Oracle final assignment of rows [a, b) of the .npy at path (child
    process of a spawn pool): labels, d1, d2."""
    path, a, b, C, live = args
    X = np.load(path, mmap_mode="r")[a:b]
    labels, _, d1, d2 = o.final_assignment(np.asarray(X), C, live)
    return a, labels.astype(np.int32), d1, d2


def final_assignment_parallel(path, m, C, live, block=500_000, workers=None):
    """o.final_assignment over all m rows of the .npy at path, cut into row
    blocks run by a spawn pool; returns (labels, d1, d2) in row order."""
    import multiprocessing as mp
    import os
    workers = workers or max(1, min(16, (os.cpu_count() or 1)))
    jobs = [(path, a, min(m, a + block), C, live) for a in range(0, m, block)]
    labels = np.empty(m, np.int32)
    d1 = np.empty(m)
    d2 = np.empty(m)
    with mp.get_context("spawn").Pool(workers) as pool:
        for a, lab, x1, x2 in pool.imap_unordered(_assign_block, jobs):
            labels[a:a + len(lab)] = lab
            d1[a:a + len(lab)] = x1
            d2[a:a + len(lab)] = x2
    return labels, d1, d2
