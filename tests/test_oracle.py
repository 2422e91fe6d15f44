"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: each checks a closed form,
an invariant, a brute-force optimum on tiny inputs, a hand-worked K-means++
example, or an independent textbook implementation.  CPU only.
"""
import itertools
import math
import os

import numpy as np
import pytest

import bminputs as bi
import oracle as o


# ------------------------------------------------------------ distances

def test_sq_distance_closed_forms():
    P = np.array([[0.0, 0.0], [3.0, 4.0], [1.0, 0.0]])
    C = np.array([[0.0, 0.0], [0.0, 1.0]])
    D = o.sq_distances(P, C)
    assert D.shape == (3, 2)
    assert D[0, 0] == 0.0 and D[1, 0] == 25.0           # 3-4-5 triangle
    assert D[2, 1] == 2.0 and D[0, 1] == 1.0            # unit vectors e1, e2
    E = np.eye(5)
    assert np.array_equal(o.sq_distances(E, E), 2.0 * (1 - np.eye(5)))


def test_sq_distance_parallel_axis_identity():
    # sum_i ||x_i - c||^2 = sum_i ||x_i - mu||^2 + m ||mu - c||^2
    rng = np.random.default_rng(0)
    X = rng.normal(size=(40, 7))
    c = rng.normal(size=(1, 7))
    mu = X.mean(axis=0, keepdims=True)
    lhs = o.sq_distances(X, c).sum()
    rhs = X.var(axis=0).sum() * 40 + 40 * float(((mu - c) ** 2).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_sq_distance_translation_and_scale():
    rng = np.random.default_rng(1)
    X, C = rng.normal(size=(9, 4)), rng.normal(size=(3, 4))
    v = rng.normal(size=(1, 4))
    assert np.allclose(o.sq_distances(X + v, C + v), o.sq_distances(X, C), rtol=1e-12)
    assert np.allclose(o.sq_distances(3 * X, 3 * C), 9 * o.sq_distances(X, C), rtol=1e-12)


def test_nearest_ties_and_degenerate_exclusion():
    P = np.array([[0.0], [1.0], [2.0]])
    C = np.array([[1.0], [1.0], [0.0], [100.0]])
    live = np.array([False, True, True, True])
    labels, d1, d2 = o.nearest(P, C, live)
    # point 1.0 ties between slots 0 and 1 but slot 0 is degenerate -> 1;
    # point 0.5-away ties resolved to the lowest live index.
    assert list(labels) == [2, 1, 1]
    assert list(d1) == [0.0, 0.0, 1.0]
    live[0] = True
    labels, _, _ = o.nearest(P, C, live)
    assert list(labels) == [2, 0, 0]       # exact tie 0 vs 1 -> lowest index


# ------------------------------------------- brute-force optimal partitions

def _partition_sse(X, labels, k):
    # within-cluster scatter via sum ||x||^2 - |X_j| ||mu_j||^2 (not the oracle route)
    tot = 0.0
    for j in range(k):
        Y = X[labels == j]
        if len(Y):
            mu = Y.sum(axis=0) / len(Y)
            tot += float((Y * Y).sum()) - len(Y) * float(mu @ mu)
    return tot


def _brute_force_optimum(X, k):
    m = X.shape[0]
    best, best_lab = math.inf, None
    for lab in itertools.product(range(k), repeat=m):
        lab = np.array(lab)
        if len(np.unique(lab)) != k:
            continue
        v = _partition_sse(X, lab, k)
        if v < best - 1e-12:
            best, best_lab = v, lab
    return best, best_lab


@pytest.mark.parametrize("m,k,seed", [(8, 2, 0), (9, 3, 1), (10, 3, 2), (12, 2, 3)])
def test_lloyd_at_brute_force_optimum_is_fixed_point(m, k, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(m, 2)) + 3 * rng.integers(0, k, size=(m, 1))
    best, lab = _brute_force_optimum(X, k)
    C = np.stack([X[lab == j].mean(axis=0) for j in range(k)])
    # the objective of the optimal centroids is the optimum
    assert o.objective(X, C, np.ones(k, bool)) == pytest.approx(best, rel=1e-9, abs=1e-12)
    res = o.lloyd(X, C, np.ones(k, bool), tol=1e-4, max_iter=300)
    assert res.iters == 1
    assert res.f == pytest.approx(best, rel=1e-9, abs=1e-12)
    assert np.allclose(res.C, C, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m,k,seed", [(9, 3, 4), (11, 2, 5), (10, 3, 6)])
def test_objective_never_below_brute_force_optimum(m, k, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(m, 3))
    best, _ = _brute_force_optimum(X, k)
    for _ in range(50):
        C = rng.normal(size=(k, 3))
        assert o.objective(X, C, np.ones(k, bool)) >= best - 1e-9
    # Lloyd from any start ends at or above the optimum
    res = o.lloyd(X, rng.normal(size=(k, 3)), np.ones(k, bool), tol=0.0)
    assert res.f >= best - 1e-9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_big_means_with_full_samples_reaches_brute_force_optimum(seed):
    # Three separated groups; s = m so every chunk sees all data.  With 30
    # chunks the K-means++ restarts reach the global optimum (expected on
    # such well-separated data).
    rng = np.random.default_rng(seed)
    m, k = 10, 3
    X = (rng.normal(size=(m, 2)) * 0.3
         + 6 * np.array([[0, 0], [1, 0], [0, 1]])[np.arange(m) % 3]).astype(np.float32)
    best, _ = _brute_force_optimum(X.astype(np.float64), k)
    draws = [bi.chunk_draws(seed, t, m, m, k) for t in range(30)]
    st, recs = o.big_means(X, k, draws)
    assert st.f_opt == pytest.approx(best, rel=1e-9)
    _, sse, _, _ = o.final_assignment(X, st.C, st.live)
    assert sse == pytest.approx(best, rel=1e-9)


# ------------------------------------------------------- Lloyd invariants

def _mixture(m=600, n=5, comps=6, seed=0):
    X, _ = bi.mixtures.isotropic_blobs(m, n, comps, seed, box=5.0)
    return X.astype(np.float64)


def test_lloyd_objective_non_increasing():
    X = _mixture()
    rng = np.random.default_rng(3)
    C = X[rng.choice(len(X), 8, replace=False)]
    res = o.lloyd(X, C, np.ones(8, bool), tol=0.0, max_iter=300)
    tr = np.array(res.f_trace)
    assert np.all(np.diff(tr) <= 1e-9 * tr[:-1])
    assert res.f == tr[-1]


def test_lloyd_fixed_point_centroid_is_member_mean():
    X = _mixture(seed=4)
    rng = np.random.default_rng(4)
    C = X[rng.choice(len(X), 7, replace=False)]
    res = o.lloyd(X, C, np.ones(7, bool), tol=0.0, max_iter=1000)
    assert res.iters < 1000
    # labels by broadcasting, means by a one-hot matrix product
    D = ((X[:, None, :] - res.C[None, :, :]) ** 2).sum(-1)
    D[:, ~res.live] = np.inf
    lab = D.argmin(1)
    M = np.zeros((len(X), 7))
    M[np.arange(len(X)), lab] = 1
    cnt = M.sum(0)
    means = (M.T @ X)[cnt > 0] / cnt[cnt > 0, None]
    assert np.allclose(res.C[cnt > 0], means, rtol=1e-10, atol=1e-10)
    # objective = sum of member distances
    assert res.f == pytest.approx(float(D.min(1).sum()), rel=1e-12)


def test_lloyd_k1_closed_form():
    X = _mixture(seed=5)
    res = o.lloyd(X, X[:1], np.ones(1, bool))
    assert np.allclose(res.C[0], X.mean(axis=0), rtol=1e-12, atol=1e-12)
    assert res.f == pytest.approx(len(X) * X.var(axis=0).sum(), rel=1e-10)


def test_lloyd_stop_rule_cases():
    X = _mixture(seed=6)
    C = X[:5].copy()
    r0 = o.lloyd(X, C, np.ones(5, bool), max_iter=0)
    assert r0.iters == 0 and np.array_equal(r0.C, C)
    r1 = o.lloyd(X, C, np.ones(5, bool), tol=1.0)      # any decrease <= f_prev
    assert r1.iters == 1
    r2 = o.lloyd(X, C, np.ones(5, bool), tol=0.0, max_iter=2)
    assert r2.iters == 2 and len(r2.f_trace) == 3


def test_lloyd_empty_cluster_becomes_degenerate():
    X = np.array([[0.0], [0.1], [5.0], [5.1]])
    C = np.array([[0.0], [5.0], [1000.0]])
    res = o.lloyd(X, C, np.ones(3, bool))
    assert list(res.live) == [True, True, False]
    assert res.f == pytest.approx(0.01, rel=1e-12)


def test_lloyd_keep_rule_leaves_an_empty_centroid_in_place():
    # R16: a centroid too far to win any row keeps its position and stays
    # live; the others follow exactly the Lloyd run without it
    X = _mixture(m=600, n=3, comps=4, seed=21)
    C0 = X[np.random.default_rng(21).choice(len(X), 4, replace=False)].copy()
    far = np.full((1, 3), 1e3)
    res = o.lloyd(X, np.vstack([C0[:2], far, C0[2:]]), np.ones(5, bool), empty="keep")
    ref = o.lloyd(X, C0, np.ones(4, bool))
    assert res.live.all()
    assert np.array_equal(res.C[2], far[0])
    assert np.allclose(np.delete(res.C, 2, axis=0), ref.C, rtol=0, atol=0)
    assert res.f == ref.f and res.iters == ref.iters
    # the default rule drops it instead
    deg = o.lloyd(X, np.vstack([C0[:2], far, C0[2:]]), np.ones(5, bool))
    assert list(deg.live) == [True, True, False, True, True]


def test_lloyd_keep_rule_never_creates_degenerate_slots():
    emptied = 0
    for seed in range(5):
        X = _mixture(m=400, n=2, comps=3, seed=30 + seed)
        # more centroids than clusters, some started on duplicated rows, so
        # that some of them lose every member along the way
        C0 = np.vstack([X[:6], X[:6]])
        res = o.lloyd(X, C0, np.ones(12, bool), empty="keep")
        assert res.live.all()
        deg = o.lloyd(X, C0, np.ones(12, bool))
        emptied += int(not deg.live.all())
    assert emptied > 0   # the cases do exercise empty clusters


def test_lloyd_matches_textbook_lloyd_at_fixed_point():
    sk = pytest.importorskip("sklearn.cluster")
    X = _mixture(m=800, n=4, comps=5, seed=7)
    C0 = X[np.random.default_rng(7).choice(len(X), 5, replace=False)]
    res = o.lloyd(X, C0, np.ones(5, bool), tol=0.0, max_iter=1000)
    km = sk.KMeans(n_clusters=5, init=C0, n_init=1, algorithm="lloyd",
                   tol=0.0, max_iter=1000).fit(X)
    assert np.allclose(res.C, km.cluster_centers_, rtol=1e-9, atol=1e-9)
    assert res.f == pytest.approx(km.inertia_, rel=1e-9)


# ------------------------------------------------------------- K-means++

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fixture(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].split()
        if line:
            out[line[0]] = [float(v) for v in line[1:]]
    return out


def test_kpp_hand_worked_example():
    # tests/golden/kpp_hand_example.txt: one slot reseeded, worked by hand
    g = _fixture("kpp_hand_example.txt")
    P = np.array(g["rows"]).reshape(-1, 1)
    live = np.array(g["live"], bool)
    C = np.zeros((len(live), 1))
    C[0, 0] = g["centroid0"][0]
    u = np.array([[0.0, 0.0, 0.0], g["uniforms"]])
    picks = []
    C2, live2 = o.kmeanspp_reseed(P, C, live, 0.0, u, 3, picks)
    assert picks[0].cands == [int(v) for v in g["candidates"]]
    assert picks[0].potentials == g["potentials"]
    assert picks[0].chosen == int(g["chosen"][0])
    assert C2[1, 0] == g["new_centroid"][0] and live2.all()


def test_kpp_first_centre_and_fill_order():
    P = np.arange(10, dtype=np.float64).reshape(10, 1) ** 2
    C = np.zeros((3, 1))
    live = np.zeros(3, bool)
    u = np.full((3, 3), 0.999)
    picks = []
    C2, live2 = o.kmeanspp_reseed(P, C, live, 0.35, u, 3, picks)
    assert C2[0, 0] == P[3, 0]                     # floor(0.35 * 10) = 3
    assert [p.slot for p in picks] == [0, 1, 2]    # ascending slots
    assert live2.all()
    # u close to 1 picks the last point with positive D^2 mass
    assert C2[1, 0] == P[9, 0]


def test_kpp_zero_potential_falls_back_to_uniform():
    P = np.ones((6, 2))
    C = np.array([[1.0, 1.0], [0.0, 0.0]])
    live = np.array([True, False])
    u = np.array([[0, 0, 0], [0.5, 0.9, 0.1]], dtype=float)
    picks = []
    C2, _ = o.kmeanspp_reseed(P, C, live, 0.0, u, 3, picks)
    assert picks[0].cands == [3, 5, 0]
    assert np.array_equal(C2[1], [1.0, 1.0])


def test_kpp_picks_follow_d2_distribution():
    # Empirical frequency of the first candidate ~ D^2 / sum D^2.
    P = np.array([[0.0], [1.0], [2.0], [4.0]])
    D2 = np.array([0.0, 1.0, 4.0, 16.0])
    counts = np.zeros(4)
    T = 3000
    for t in range(T):
        u = bi.kpp_uniforms(0, t, 2, 3)
        picks = []
        o.kmeanspp_reseed(P, np.zeros((2, 1)), np.array([True, False]), 0.0, u, 3, picks)
        counts[picks[0].cands[0]] += 1
    expected = T * D2 / D2.sum()
    assert counts[0] == 0
    chi2 = ((counts[1:] - expected[1:]) ** 2 / expected[1:]).sum()
    assert chi2 < 20   # 2 dof


def test_k_equals_s_distinct_points_gives_zero_sse():
    X = np.random.default_rng(8).normal(size=(12, 3)).astype(np.float32)
    draws = [bi.chunk_draws(1, 0, 12, 12, 12)]
    st, recs = o.big_means(X, 12, draws)
    assert st.f_opt == 0.0 and st.live.all()


# ------------------------------------------------------------- Big-means

def test_big_means_incumbent_non_increasing_and_keep_best_rule():
    X = bi.mixtures.blobs_2d(m=4000)
    draws = [bi.chunk_draws(0, t, 4000, 400, 10) for t in range(12)]
    st, recs = o.big_means(X, 10, draws)
    f_opt = math.inf
    for r in recs:
        assert r.accepted == (r.f_chunk < f_opt)
        if r.accepted:
            f_opt = r.f_chunk
    assert st.f_opt == f_opt
    assert recs[0].accepted


def test_keep_best_is_strict_on_ties():
    # s = m: every chunk is the whole data; from a converged incumbent the
    # next chunk reproduces the same objective and must not replace it.
    X = _mixture(m=200, n=2, comps=3, seed=9).astype(np.float32)
    d = bi.chunk_draws(0, 0, 200, 200, 3)
    st, recs = o.big_means(X, 3, [d, d, d], tol=0.0, max_iter=1000)
    assert recs[0].accepted
    assert not recs[1].accepted and not recs[2].accepted
    assert recs[1].f_chunk == recs[0].f_chunk


def test_degenerate_incumbent_slots_are_reseeded_next_chunk():
    X = _mixture(m=300, n=2, comps=3, seed=10).astype(np.float32)
    st = o.BigMeansState(4, 2)
    st.C[:2] = X[:2]
    st.live[:2] = True
    st.f_opt = 1e30
    idx, uf, u = bi.chunk_draws(2, 0, 300, 150, 4)
    rec = o.big_means_chunk(X, st, idx, uf, u)
    assert [p.slot for p in rec.picks] == [2, 3]
    assert rec.accepted


def test_n_d_counter_convention():
    X = bi.mixtures.blobs_2d(m=2000)
    d = bi.chunk_draws(0, 0, 2000, 500, 10)
    st, recs = o.big_means(X, 10, [d])
    r = recs[0]
    # all slots degenerate: s for the first centre, 3 s per further slot,
    # then s x 10 per assignment step (no centroid emptied on blobs).
    assert r.lloyd.live.all()
    assert r.n_d == 500 + 9 * 3 * 500 + (r.iters + 1) * 500 * 10


def test_workers_with_one_worker_are_sequential_big_means():
    # both parallel modes with a single worker reduce to Alg. 1
    X, _ = bi.mixtures.isotropic_blobs(3000, 3, 6, 4)
    k, s, T = 5, 400, 6
    draws_of = lambda t: bi.chunk_draws(4, t, 3000, s, k)
    ref, recs = o.big_means(X, k, [draws_of(t) for t in range(T)])
    for mode in ("competitive", "collective"):
        st, recs_w = o.big_means_workers(X, k, draws_of, 1, T, mode)
        assert st.f_opt == ref.f_opt and np.array_equal(st.C, ref.C)
        assert [r.accepted for r in recs_w] == [r.accepted for r in recs]


def test_competitive_workers_are_independent_runs():
    # mode 2: worker w runs Alg. 1 on chunks w, w + W, ...; the best wins
    X, _ = bi.mixtures.isotropic_blobs(3000, 3, 6, 5)
    k, s, W, R = 5, 300, 3, 4
    draws_of = lambda t: bi.chunk_draws(5, t, 3000, s, k)
    st, _ = o.big_means_workers(X, k, draws_of, W, R, "competitive")
    runs = [o.big_means(X, k, [draws_of(r * W + w) for r in range(R)])[0] for w in range(W)]
    best = min(range(W), key=lambda w: (runs[w].f_opt, w))
    assert st.f_opt == runs[best].f_opt and np.array_equal(st.C, runs[best].C)


def test_collective_incumbent_never_worsens():
    X, _ = bi.mixtures.isotropic_blobs(3000, 3, 6, 6)
    k, s, W = 5, 300, 3
    draws_of = lambda t: bi.chunk_draws(6, t, 3000, s, k)
    prev = math.inf
    for R in range(1, 5):
        st, _ = o.big_means_workers(X, k, draws_of, W, R, "collective")
        assert st.f_opt <= prev
        prev = st.f_opt


def test_forgy_reseed_picks_uniform_rows_in_slot_order():
    P = np.arange(20, dtype=np.float64).reshape(10, 2)
    C = np.full((4, 2), -7.0)
    live = np.array([False, True, False, False])
    u = np.array([[0.05, 0.9, 0.9], [0.5, 0.5, 0.5], [0.999, 0.1, 0.1], [0.31, 0.0, 0.0]])
    C2, live2 = o.forgy_reseed(P, C, live, u)
    assert live2.all()
    assert np.array_equal(C2[0], P[0]) and np.array_equal(C2[2], P[9])
    assert np.array_equal(C2[3], P[3]) and np.array_equal(C2[1], C[1])   # live slot kept


def test_forgy_big_means_counts_no_reseed_distances():
    X, _ = bi.mixtures.isotropic_blobs(2000, 3, 5, 8)
    k, s = 4, 500
    draws = [bi.chunk_draws(8, t, 2000, s, k) for t in range(3)]
    st, recs = o.big_means(X, k, draws, init="forgy")
    assert st.live.all() and math.isfinite(st.f_opt)
    assert recs[0].n_d == recs[0].lloyd.n_d              # Forgy evaluates no distances


def test_oracle_reproduces_its_recorded_runs():
    # tests/golden/oracle_small_runs.json was written by
    # tests/golden/make_golden.py from the oracle alone; a change of the
    # oracle's arithmetic shows up here and must be justified by the paper
    import importlib.util
    import json
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    rec = json.load(open(os.path.join(GOLDEN, "oracle_small_runs.json")))
    assert len(rec["cases"]) == len(mg.CASES)
    for case in rec["cases"]:
        got = mg.run(case["m"], case["n"], case["k"], case["s"], case["chunks"],
                     case["components"], case["seed"], case["box"])
        want = case["result"]
        assert got["live"] == want["live"] and got["accepted"] == want["accepted"]
        assert got["iters"] == want["iters"] and got["labels_sum"] == want["labels_sum"]
        assert got["f_opt"] == pytest.approx(want["f_opt"], rel=1e-12)
        assert got["sse"] == pytest.approx(want["sse"], rel=1e-12)
        assert np.allclose(got["C"], want["C"], rtol=1e-12, atol=1e-12)
