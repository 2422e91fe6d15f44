"""Pins of the oracle's decision following (reading R17) and of the search
that uses it (tests/parity_follow.py), on the CPU.

Each exempt decision is built by hand so that both outcomes are known in
closed form; taking the other outcome must give exactly the other one, and
without flips the oracle must be unchanged.
"""
import numpy as np

import bminputs as bi
import oracle as o
import parity_follow as pf


def _state(C, live, f_opt=np.inf):
    st = o.BigMeansState(*np.asarray(C).shape)
    st.C = np.asarray(C, np.float64).copy()
    st.live = np.asarray(live, bool).copy()
    st.f_opt = f_opt
    return st


def test_decisions_without_flips_change_nothing():
    m, n, k, s = 3000, 5, 6, 800
    X, _ = bi.mixtures.isotropic_blobs(m, n, k, 11)
    draws = [bi.chunk_draws(11, t, m, s, k) for t in range(3)]
    st0, recs0 = o.big_means(X, k, draws)
    d = o.Decisions()
    st1, recs1 = o.big_means(X, k, draws, decisions=d)
    assert np.array_equal(st0.C, st1.C) and np.array_equal(st0.live, st1.live)
    assert st0.f_opt == st1.f_opt
    assert [r.iters for r in recs0] == [r.iters for r in recs1]
    for key, margin in d.met:          # every recorded decision lies in its band
        assert margin >= 0


def test_label_flip_hand_example():
    """1-D rows 0, 2, 1 and centroids 0, 2: row 2 is equidistant (d = 1).
    Lowest index: c = (0.5, 2); the other outcome: c = (0, 1.5); both end at
    f = 0.5 after two update steps."""
    P = np.array([[0.0], [2.0], [1.0]])
    C0 = np.array([[0.0], [2.0]])
    live = np.array([True, True])
    a = o.lloyd(P, C0, live)
    assert np.allclose(a.C[:, 0], [0.5, 2.0]) and a.f == 0.5 and a.iters == 2
    d = o.Decisions([("label", 0, 0, 2)])
    b = o.lloyd(P, C0, live, decisions=d, t=0)
    assert np.allclose(b.C[:, 0], [0.0, 1.5]) and b.f == 0.5 and b.iters == 2
    assert (("label", 0, 0, 2), 0.0) in d.met


def test_kpp_target_flip_takes_the_row_across_the_boundary():
    """D^2 = 1, 1, 2 to the live centre (0, 0); prefix 1, 2, 4; u = 0.5 puts
    the target 2 exactly on the boundary between rows 1 and 2: the rule picks
    row 2, the other outcome row 1."""
    P = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    C = np.array([[0.0, 0.0], [9.0, 9.0]])
    live = np.array([True, False])
    u = np.array([[0.5], [0.5]])
    Ca, _ = o.kmeanspp_reseed(P, C, live, 0.0, u, trials=1)
    assert np.array_equal(Ca[1], P[2])
    d = o.Decisions([("kpp_target", 0, 1, 0)])
    Cb, _ = o.kmeanspp_reseed(P, C, live, 0.0, u, trials=1, decisions=d, t=0)
    assert np.array_equal(Cb[1], P[1])
    assert d.met == [(("kpp_target", 0, 1, 0), 0.0)]


def test_kpp_best_flip_takes_the_other_equal_potential():
    """Rows -1, 1, 0 with the centre at 0: candidates -1 (u = 0.25) and 1
    (u = 0.75) both leave potential 1; the lowest trial wins, the other
    outcome takes the second."""
    P = np.array([[-1.0], [1.0], [0.0]])
    C = np.array([[0.0], [5.0]])
    live = np.array([True, False])
    u = np.array([[0.25, 0.75], [0.25, 0.75]])
    picks = []
    Ca, _ = o.kmeanspp_reseed(P, C, live, 0.0, u, trials=2, picks=picks)
    assert picks[0].potentials == [1.0, 1.0] and Ca[1, 0] == -1.0
    d = o.Decisions([("kpp_best", 0, 1)])
    Cb, _ = o.kmeanspp_reseed(P, C, live, 0.0, u, trials=2, decisions=d, t=0)
    assert Cb[1, 0] == 1.0


def test_keep_flip_accepts_an_equal_objective():
    P = np.array([[0.0], [2.0], [1.0]])
    st = _state([[0.0], [2.0]], [True, True], f_opt=0.5)
    rec = o.big_means_chunk(P, st.copy(), [0, 1, 2], 0.0, np.zeros((2, 3)))
    assert rec.f_chunk == 0.5 and not rec.accepted            # strict: a tie keeps
    d = o.Decisions([("keep", 0)])
    st2 = st.copy()
    rec2 = o.big_means_chunk(P, st2, [0, 1, 2], 0.0, np.zeros((2, 3)), decisions=d)
    assert rec2.accepted and st2.f_opt == 0.5


def test_stop_flip_reverses_a_test_at_its_threshold():
    m, n, k, s = 2000, 3, 5, 1000
    X, _ = bi.mixtures.isotropic_blobs(m, n, k, 3)
    P = X[:s].astype(np.float64)
    C0 = P[:k].copy()
    live = np.ones(k, bool)
    free = o.lloyd(P, C0, live, tol=0.0)
    f0, f1 = free.f_trace[0], free.f_trace[1]
    tol = (f0 - f1) / f0                 # step 1 sits on the threshold
    d = o.Decisions()
    a = o.lloyd(P, C0, live, tol=tol, decisions=d)
    keys = [k_ for k_, _ in d.met if k_[0] == "stop"]
    assert ("stop", 0, 1) in keys
    b = o.lloyd(P, C0, live, tol=tol, decisions=o.Decisions([("stop", 0, 1)]))
    assert sorted([a.iters, b.iters])[0] == 1 and a.iters != b.iters


def test_follow_chunk_finds_a_planted_decision():
    """The 'GPU' outcome here is the oracle's own run with one exempt row
    taking its other label; the search must name exactly that decision."""
    P = np.array([[0.0], [2.0], [1.0]], np.float32)
    st = _state([[0.0], [2.0]], [True, True])
    planted = st.copy()
    rec = o.big_means_chunk(P, planted, [0, 1, 2], 0.0, np.zeros((2, 3)),
                            decisions=o.Decisions([("label", 0, 0, 2)]))
    obs = {"accepted": rec.accepted, "iters": rec.iters, "f_opt": planted.f_opt,
           "C": planted.C, "live": planted.live}
    hit = pf.follow_chunk(P, st, ([0, 1, 2], 0.0, np.zeros((2, 3))), 0, obs)
    assert hit is not None and hit[2] == (("label", 0, 0, 2),)
    assert np.allclose(hit[0].C[:, 0], [0.0, 1.5])
    # and the unflipped outcome is not accepted as a match
    plain = st.copy()
    rec0 = o.big_means_chunk(P, plain, [0, 1, 2], 0.0, np.zeros((2, 3)))
    assert not pf.chunk_matches(plain, rec0, obs)
