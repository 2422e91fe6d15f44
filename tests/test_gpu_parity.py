"""GPU parity of every step of the Big-means hot path against the FP64 oracle.

Every call goes through the C ABI (libbigmeans.so via the ctypes binding).
Inputs are seeded; the oracle and the GPU consume the same Philox draws (the
CUDA library regenerates them on the device; test_draw_* pins that equality
bit for bit).

Trajectory-level cases (Lloyd runs, chunks, whole runs) are "decisive": the
oracle's own run has no decision inside the exemption bands -- no row whose
top-two distances are within 1e-5 relative at any assignment step, no stop
test or keep-the-best comparison within 1e-6 relative of its threshold, no
K-means++ inverse-CDF target within 5e-8 * sum(D^2) of a prefix boundary and
no two distinct candidate potentials within 1e-6 relative.  Each such test
asserts that precondition from the oracle's record, then demands agreement.
"""
import math

import numpy as np
import pytest

import bminputs as bi
import oracle as o
from gpu_helpers import (CEN_REL, OBJ_REL, centroids_close, dev, host,
                         labels_match, rel, require_gpu, torch)

pytestmark = pytest.mark.gpu

KPP_BAND = 5e-8


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


def _margins(rec):
    pm = min([p.boundary_margin for p in rec.picks] or [math.inf])
    pg = math.inf
    for p in rec.picks:
        pots = sorted(set(p.potentials))
        if len(pots) > 1:
            pg = min(pg, (pots[1] - pots[0]) / pots[0])
    return dict(gap=rec.lloyd.min_gap, stop=rec.lloyd.stop_margin,
                keep=rec.keep_margin, kpp=pm, pot=pg)


def _assert_decisive(recs):
    for r in recs:
        mg = _margins(r)
        assert mg["gap"] >= 1e-5 and mg["stop"] >= 1e-6 and mg["keep"] >= 1e-6 \
            and mg["kpp"] >= KPP_BAND and mg["pot"] >= 1e-6, \
            "case not decisive at chunk %d: %r" % (r.t, mg)


# ------------------------------------------------------------ a1: sample draw

@pytest.mark.parametrize("m,s,seed,t", [
    (20000, 2000, 0, 0), (20000, 2000, 0, 7), (1_000_000, 50_000, 0, 3),
    (100, 80, 7, 1), (33, 33, 1, 0), (1000, 1, 2, 3), (37, 18, 3, 2),
    (64, 33, 5, 9), (10_000_000, 50_000, 0, 0), (2_000_000, 50_000, 11, 99)])
def test_draw_matches_generator_bit_exact(bm, m, s, seed, t):
    idx = torch.empty(s, dtype=torch.int32, device="cuda:0")
    bm.bm_draw_chunk(m, s, seed, t, idx)
    ref = bi.chunk_indices(seed, t, m, s)
    assert np.array_equal(host(idx).astype(np.int64), ref)


def test_draw_repeated_calls_are_identical(bm):
    a = torch.empty(5000, dtype=torch.int32, device="cuda:0")
    b = torch.empty_like(a)
    bm.bm_draw_chunk(200_000, 5000, 4, 12, a)
    bm.bm_draw_chunk(200_000, 5000, 4, 12, b)
    assert torch.equal(a, b)


# ----------------------------------------------------------- a1: gather

@pytest.mark.parametrize("m,n,s", [(3000, 1, 700), (5000, 2, 2000), (4099, 28, 1111),
                                   (2500, 33, 999), (1200, 128, 300), (300, 384, 77)])
def test_gather_bit_exact(bm, m, n, s):
    X = np.random.default_rng(n).normal(size=(m, n)).astype(np.float32)
    idx = bi.chunk_indices(1, 0, m, s)
    P = torch.empty((s, n), dtype=torch.float32, device="cuda:0")
    bm.bm_gather(dev(X), m, n, dev(idx.astype(np.int32)), s, P)
    assert np.array_equal(host(P), X[idx])


# ------------------------------------------------------ a3/a8: assignment

ASSIGN_CASES = [(5000, 2, 10, 0), (4097, 28, 25, 1), (3001, 128, 50, 2),
                (2000, 1, 3, 3), (1000, 33, 100, 4), (777, 127, 7, 5),
                (64, 5, 1, 6), (10_000, 16, 128, 7), (513, 384, 20, 8),
                (512, 12, 6, 9), (204_800, 7, 9, 10), (300_001, 28, 25, 11),
                (100_003, 32, 40, 12)]


@pytest.mark.parametrize("m,n,k,seed", ASSIGN_CASES)
def test_assign_rows_matches_oracle(bm, m, n, k, seed):
    X, _ = bi.mixtures.isotropic_blobs(m, n, max(k, 2), seed, box=5.0)
    rng = np.random.default_rng(seed)
    C = (X[rng.choice(m, k, replace=False)]
         + rng.normal(scale=0.1, size=(k, n))).astype(np.float32)
    live = np.ones(k, bool)
    if k > 3:
        live[rng.choice(k, k // 4, replace=False)] = False
    labels = torch.empty(m, dtype=torch.int32, device="cuda:0")
    dmin = torch.empty(m, dtype=torch.float32, device="cuda:0")
    sse = bm.bm_assign_rows(dev(X), m, n, dev(C), dev(live.astype(np.uint8)), k,
                            labels, dmin)
    ref_lab, d1, d2 = o.nearest(X, C, live)
    bad, ties = labels_match(host(labels), ref_lab, d1, d2)
    assert bad == 0, "%d label mismatches outside the tie band (%d ties)" % (bad, ties)
    tol = (n + 2) * 2.0 ** -24
    np.testing.assert_allclose(host(dmin), d1, rtol=tol, atol=1e-30)
    assert rel(sse, float(d1.sum())) <= OBJ_REL


@pytest.mark.parametrize("n_extra", [0, 40])   # np path and generic path
def test_assign_exact_ties_take_lowest_index(bm, n_extra):
    X = np.array([[0.0, 0.0], [0.5, 0.0], [9.0, 9.0], [1.0, 0.0]], np.float32)
    C = np.array([[0.5, 1.0], [0.5, -1.0], [9.0, 9.0], [9.0, 9.0]], np.float32)
    X = np.pad(X, ((0, 0), (0, n_extra)))
    C = np.pad(C, ((0, 0), (0, n_extra)))
    n = X.shape[1]
    labels = torch.empty(4, dtype=torch.int32, device="cuda:0")
    # rows 0, 1, 3 tie slots 0 and 1 exactly; row 2 ties slots 2 and 3
    bm.bm_assign_rows(dev(X), 4, n, dev(C), dev(np.ones(4, np.uint8)), 4, labels)
    assert list(host(labels)) == [0, 0, 2, 0]
    # with slot 0 degenerate the ties go to the next live slot
    bm.bm_assign_rows(dev(X), 4, n, dev(C), dev(np.array([0, 1, 0, 1], np.uint8)), 4,
                      labels)
    assert list(host(labels)) == [1, 1, 3, 1]


# --------------------------------------------------------- a2: K-means++

KPP_CASES = [  # (m, n, k, s, seed, t, live_fraction)
    (20000, 2, 10, 2000, 0, 0, 0.0),
    (20000, 2, 10, 2000, 0, 3, 0.5),
    (8000, 28, 25, 5000, 1, 0, 0.0),
    (6000, 128, 50, 3000, 2, 0, 0.0),
    (1500, 33, 7, 500, 3, 1, 0.3),
    (4000, 5, 13, 1000, 4, 2, 0.8),
]


@pytest.mark.parametrize("m,n,k,s,seed,t,frac", KPP_CASES)
def test_kpp_reseed_matches_oracle(bm, m, n, k, s, seed, t, frac):
    X, _ = bi.mixtures.isotropic_blobs(m, n, max(k, 2), seed)
    idx, uf, u = bi.chunk_draws(seed, t, m, s, k)
    P = X[idx]
    rng = np.random.default_rng(seed + 100)
    live = rng.random(k) < frac
    C = np.zeros((k, n), np.float32)
    C[live] = P[rng.choice(s, int(live.sum()), replace=False)]
    picks = []
    C_ref, live_ref = o.kmeanspp_reseed(P, C, live, uf, u, 3, picks)
    for p in picks:
        assert p.boundary_margin >= KPP_BAND, "not decisive: %r" % p.boundary_margin
        pots = sorted(set(p.potentials))
        assert len(pots) < 2 or (pots[1] - pots[0]) / pots[0] >= 1e-6
    Cd = dev(C)
    md = dev(live.astype(np.uint8))
    bm.bm_kpp_reseed(dev(P), s, n, k, Cd, md, seed, t, 3)
    assert np.array_equal(host(md).astype(bool), live_ref)
    # reseeded centroids are copies of sample rows: bit-exact
    assert np.array_equal(host(Cd).astype(np.float64), C_ref)


def test_kpp_all_identical_points_uniform_fallback(bm):
    s, n, k = 300, 3, 4
    P = np.full((s, n), 2.5, np.float32)
    C = np.zeros((k, n), np.float32)
    live = np.zeros(k, bool)
    uf, u = bi.kpp_uniform_first(9, 0), bi.kpp_uniforms(9, 0, k)
    C_ref, live_ref = o.kmeanspp_reseed(P, C, live, uf, u)
    Cd, md = dev(C), dev(live.astype(np.uint8))
    bm.bm_kpp_reseed(dev(P), s, n, k, Cd, md, 9, 0, 3)
    assert host(md).all() and np.array_equal(host(Cd).astype(np.float64), C_ref)


# ------------------------------------------------------------ a3-a6: Lloyd

LLOYD_CASES = [  # (m, n, k, s, seed, t, max_iter, tol)
    (20000, 2, 10, 2000, 0, 0, 300, 1e-4),
    (20000, 2, 10, 2000, 1, 0, 300, 1e-5),
    (30000, 28, 25, 6000, 6, 0, 300, 1e-4),
    (6000, 128, 50, 3000, 3, 0, 300, 1e-4),
    (3000, 33, 9, 1111, 4, 0, 2, 0.0),
    (3000, 7, 1, 999, 5, 0, 300, 1e-4),
    (5000, 3, 20, 1500, 6, 0, 1, 1e-4),
    (5000, 3, 20, 1500, 6, 0, 0, 1e-4),
]


@pytest.mark.parametrize("m,n,k,s,seed,t,max_iter,tol", LLOYD_CASES)
def test_lloyd_matches_oracle(bm, m, n, k, s, seed, t, max_iter, tol):
    X, _ = bi.mixtures.isotropic_blobs(m, n, max(2 * k, 2), seed, box=6.0)
    idx, uf, u = bi.chunk_draws(seed, t, m, s, k)
    P = X[idx]
    C0, live0 = o.kmeanspp_reseed(P, np.zeros((k, n)), np.zeros(k, bool), uf, u)
    res = o.lloyd(P, C0, live0, tol=tol, max_iter=max_iter)
    assert res.min_gap >= 1e-5 and res.stop_margin >= 1e-6, \
        "not decisive: gap %g stop %g" % (res.min_gap, res.stop_margin)
    Cd = dev(C0.astype(np.float32))
    md = dev(live0.astype(np.uint8))
    f, iters = bm.bm_lloyd(dev(P), s, n, k, Cd, md, max_iter, tol)
    assert iters == res.iters
    assert np.array_equal(host(md).astype(bool), res.live)
    assert rel(f, res.f) <= OBJ_REL
    assert centroids_close(host(Cd), res.C, res.live) <= CEN_REL


def test_lloyd_empty_cluster_becomes_degenerate(bm):
    P = np.array([[0.0], [0.1], [5.0], [5.1]], np.float32)
    C = np.array([[0.0], [5.0], [1000.0]], np.float32)
    Cd, md = dev(C), dev(np.ones(3, np.uint8))
    f, iters = bm.bm_lloyd(dev(P), 4, 1, 3, Cd, md)
    assert list(host(md)) == [1, 1, 0]
    assert rel(f, 0.01) <= 1e-6


# ------------------------------------------------------ a1-a7: whole chunks

def _run_gpu_chunks(bm, X, cfg, T):
    ctx = bm.bm_create(cfg, dev(X))
    try:
        rep = bm.bm_fit_chunk(ctx, T)
        k, n = cfg.k, cfg.n
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt, tc = bm.bm_get_state(ctx, C, mask)
    finally:
        bm.bm_destroy(ctx)
    return rep, C, mask.astype(bool), f_opt


def test_blobs_2d_full_run_free_running(bm):
    """m = 20,000, n = 2, k = 10, s = 2,000, 20 chunks, seed 0, then final assignment."""
    m, n, k, s, T, seed = 20000, 2, 10, 2000, 20, 0
    X = bi.mixtures.blobs_2d(seed)
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    st, recs = o.big_means(X, k, draws)
    _assert_decisive(recs)
    Xd = dev(X)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed)
    ctx = bm.bm_create(cfg, Xd)
    try:
        rep = bm.bm_fit_chunk(ctx, T)
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt = bm.bm_objective(ctx, C, mask)
        labels = torch.empty(m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, labels)
    finally:
        bm.bm_destroy(ctx)
    assert rep["chunks"] == T
    assert rep["accepted"] == sum(r.accepted for r in recs)
    assert rep["lloyd_iters"] == sum(r.iters for r in recs)
    assert np.array_equal(mask.astype(bool), st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
    A, sse_ref, d1, d2 = o.final_assignment(X, st.C, st.live)
    bad, _ = labels_match(host(labels), A, d1, d2)
    assert bad == 0
    assert rel(sse, sse_ref) <= OBJ_REL
    assert rep["n_d"] == sum(r.n_d for r in recs)   # Sec. 5 counter


@pytest.mark.parametrize("seed,chunks", [(6, (0, 1, 3, 5, 6, 7))])
def test_hepmass_like_full_size_chunks_teacher_forced(bm, seed, chunks):
    """m = 1e6, n = 28, k = 25, s = 50,000: each chunk starts from the oracle's
    incumbent (set through bm_set_state) and must end at the oracle's."""
    m, n, k, s = 1_000_000, 28, 25, 50_000
    X = bi.mixtures.hepmass_like(0)
    Xd = dev(X)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed)
    ctx = bm.bm_create(cfg, Xd)
    st = o.BigMeansState(k, n)
    try:
        for t in range(max(chunks) + 1):
            before = st.copy()
            idx, uf, u = bi.chunk_draws(seed, t, m, s, k)
            rec = o.big_means_chunk(X, st, idx, uf, u, t=t)
            if t not in chunks:
                continue
            _assert_decisive([rec])
            Cb = before.C.astype(np.float32)
            bm.bm_set_state(ctx, Cb, before.live.astype(np.uint8), before.f_opt, t)
            rep = bm.bm_fit_chunk(ctx, 1)
            C = np.zeros((k, n), np.float32)
            mask = np.zeros(k, np.uint8)
            f_opt, tc = bm.bm_get_state(ctx, C, mask)
            assert tc == t + 1
            assert rep["accepted"] == int(rec.accepted)
            assert rep["lloyd_iters"] == rec.iters
            assert np.array_equal(mask.astype(bool), st.live)
            assert rel(f_opt, st.f_opt) <= OBJ_REL
            assert centroids_close(C, st.C, st.live) <= CEN_REL
        # final assignment at full size against the oracle's incumbent
        bm.bm_set_state(ctx, st.C.astype(np.float32), st.live.astype(np.uint8), st.f_opt, 0)
        labels = torch.empty(m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, labels)
    finally:
        bm.bm_destroy(ctx)
    C32 = st.C.astype(np.float32)
    A, sse_ref, d1, d2 = o.final_assignment(X, C32, st.live)
    bad, _ = labels_match(host(labels), A, d1, d2)
    assert bad == 0
    assert rel(sse, sse_ref) <= OBJ_REL


# ------------------------------------------------- determinism, checkpoint

def test_runs_are_bitwise_deterministic_and_resumable(bm):
    m, n, k, s = 30000, 12, 16, 3000
    X, _ = bi.mixtures.isotropic_blobs(m, n, 20, 3)
    Xd = dev(X)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=42)

    def state(ctx):
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f, t = bm.bm_get_state(ctx, C, mask)
        return C, mask, f, t

    a = bm.bm_create(cfg, Xd)
    bm.bm_fit_chunk(a, 8)
    S8 = state(a)
    bm.bm_reset(a)
    bm.bm_fit_chunk(a, 8)
    S8b = state(a)
    bm.bm_reset(a)
    bm.bm_fit_chunk(a, 4)
    S4 = state(a)
    bm.bm_destroy(a)
    b = bm.bm_create(cfg, Xd)
    bm.bm_set_state(b, S4[0], S4[1], S4[2], S4[3])
    bm.bm_fit_chunk(b, 4)
    S8c = state(b)
    bm.bm_destroy(b)
    for other in (S8b, S8c):
        assert np.array_equal(S8[0], other[0]) and np.array_equal(S8[1], other[1])
        assert S8[2] == other[2] and S8[3] == other[3]


def test_fit_host_matches_device_path(bm):
    m, n, k, s, T = 20000, 2, 10, 2000, 6
    X = bi.mixtures.blobs_2d(0)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=0)
    C = np.zeros((k, n), np.float32)
    mask = np.zeros(k, np.uint8)
    lab = np.zeros(m, np.int32)
    sse, rep = bm.bm_fit_host(cfg, X, T, C, mask, lab)
    rep2, C2, mask2, f2 = _run_gpu_chunks(bm, X, cfg, T)
    assert np.array_equal(C, C2) and np.array_equal(mask.astype(bool), mask2)
    assert rep["f_opt"] == f2
    ref_lab, sse_ref, d1, d2 = o.final_assignment(X, C, mask.astype(bool))
    assert labels_match(lab, ref_lab, d1, d2)[0] == 0
    assert rel(sse, sse_ref) <= OBJ_REL


@pytest.mark.parametrize("m,n,k,s,T,prec", [
    (2_000_000, 28, 25, 50_000, 6, 0),     # row-in-register gather
    (1_000_000, 40, 20, 20_000, 4, 0),     # tiled FP32 gather
    (1_000_000, 128, 50, 20_000, 4, 3),    # tensor-core chunk kernel gather
])
def test_fit_host_pinned_overlap_equals_device_path(bm, m, n, k, s, T, prec):
    # pinned host rows: chunks that start while the copy to the device is in
    # flight gather from host memory; every result must equal the path that
    # runs on a device copy of X, bit for bit, whichever source each CTA used
    X = bi.mixtures.isotropic_blobs_device(m, n, 60, 5, device="cuda:0").cpu().numpy()
    Xh = torch.from_numpy(X).pin_memory()
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=9, precision=prec)
    C = np.zeros((k, n), np.float32)
    mask = np.zeros(k, np.uint8)
    lab = torch.empty(m, dtype=torch.int32).pin_memory()
    bm.bm_fit_host(cfg, Xh.data_ptr(), 1, C, mask, lab.data_ptr())   # warm: pool, modules
    # a competing host-to-device copy keeps the copy engines busy, so the
    # first chunks of the measured call are likely to start before X lands
    big = torch.empty(256 << 20, dtype=torch.float32).pin_memory()
    side = torch.cuda.Stream()
    busy = torch.empty_like(big, device="cuda:0")
    with torch.cuda.stream(side):
        busy.copy_(big, non_blocking=True)
    sse, rep = bm.bm_fit_host(cfg, Xh.data_ptr(), T, C, mask, lab.data_ptr())
    torch.cuda.synchronize()
    assert rep["host_gathers"] >= 0
    Xd = dev(X)
    ctx = bm.bm_create(cfg, Xd)
    try:
        rep2 = bm.bm_fit_chunk(ctx, T)
        C2 = np.zeros((k, n), np.float32)
        mask2 = np.zeros(k, np.uint8)
        f2, _ = bm.bm_get_state(ctx, C2, mask2)
        lab2 = torch.empty(m, dtype=torch.int32, device="cuda:0")
        sse2 = bm.bm_assign(ctx, lab2)
    finally:
        bm.bm_destroy(ctx)
    print("host_gathers", rep["host_gathers"])
    assert rep2["host_gathers"] == 0
    assert np.array_equal(C, C2) and np.array_equal(mask, mask2)
    assert rep["f_opt"] == f2 and rep["accepted"] == rep2["accepted"]
    assert rep["lloyd_iters"] == rep2["lloyd_iters"]
    assert np.array_equal(lab.numpy(), host(lab2)) and sse == sse2


@pytest.mark.parametrize("m,n,k,s,prec,seed", [
    (20_000, 6, 5, 3000, 0, 40),    # row-in-register kernel
    (8000, 40, 6, 2500, 0, 41),     # tiled FP32 kernel
    (6000, 64, 7, 3000, 3, 42),     # tensor-core chunk kernel
])
def test_keep_rule_leaves_an_empty_centroid_live_in_place(bm, m, n, k, s, prec, seed):
    # an incumbent with one centroid far from every row: under BM_EMPTY_KEEP it
    # loses all members, stays live and does not move (R16); every chunk must
    # match the oracle run with the same rule
    X, _ = bi.mixtures.isotropic_blobs(m, n, k + 2, seed, box=8.0)
    rng = np.random.default_rng(seed)
    C = X[rng.choice(m, k, replace=False)].astype(np.float32)
    C[k // 2] = 1e3
    T = 2
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    st = o.BigMeansState(k, n)
    st.C = C.astype(np.float64)
    st.live = np.ones(k, bool)
    st.f_opt = 1e30
    st, recs = o.big_means(X, k, draws, state=st, empty="keep")
    _assert_decisive(recs)
    assert st.live.all() and np.array_equal(st.C[k // 2], C[k // 2].astype(np.float64))
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec,
                               empty=bm.BM_EMPTY_KEEP)
    ctx = bm.bm_create(cfg, dev(X))
    try:
        bm.bm_set_state(ctx, C, np.ones(k, np.uint8), 1e30, 0)
        rep = bm.bm_fit_chunk(ctx, T)
        C2 = np.zeros((k, n), np.float32)
        mask2 = np.zeros(k, np.uint8)
        f2, _ = bm.bm_get_state(ctx, C2, mask2)
    finally:
        bm.bm_destroy(ctx)
    assert rep["accepted"] == sum(r.accepted for r in recs)
    assert rep["lloyd_iters"] == sum(r.iters for r in recs)
    assert np.array_equal(mask2.astype(bool), st.live)
    assert np.array_equal(C2[k // 2], C[k // 2])
    assert rel(f2, st.f_opt) <= OBJ_REL
    assert centroids_close(C2, st.C, st.live) <= CEN_REL


# ---------------------------------------------------------------- edges

@pytest.mark.parametrize("m,n,k,s,seed,T", [
    (500, 3, 4, 500, 0, 1),      # s = m: the sample is all of X (complement draw)
    (900, 2, 9, 9, 1, 3),        # k = s
    (2000, 1, 3, 700, 2, 3),     # n = 1
    (1200, 40, 1, 400, 3, 3),    # k = 1, generic path
    (3000, 64, 33, 1000, 4, 3),  # k just above one lane group
])
def test_edge_shapes_full_chunks(bm, m, n, k, s, seed, T):
    X, _ = bi.mixtures.isotropic_blobs(m, n, max(k, 2), seed, box=8.0)
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    st, recs = o.big_means(X, k, draws)
    _assert_decisive(recs)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed)
    rep, C, mask, f_opt = _run_gpu_chunks(bm, X, cfg, T)
    assert np.array_equal(mask, st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
    assert rep["accepted"] == sum(r.accepted for r in recs)


def test_identical_points(bm):
    m, n, k, s = 400, 2, 3, 100
    X = np.full((m, n), -1.25, np.float32)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=5)
    rep, C, mask, f_opt = _run_gpu_chunks(bm, X, cfg, 2)
    draws = [bi.chunk_draws(5, t, m, s, k) for t in range(2)]
    st, recs = o.big_means(X, k, draws)
    assert f_opt == 0.0 == st.f_opt
    assert np.array_equal(mask, st.live)


@pytest.mark.parametrize("prec", [0, 2])
def test_context_keeps_a_temporary_dataset_alive(bm, prec):
    # the context borrows X; a temporary tensor handed to bm_create stays
    # referenced by the binding, so later allocations of the same size (the
    # labels, scratch filled with garbage) cannot take its memory
    m, n, k, s, T, seed = 5432, 2 if prec == 0 else 100, 3, 2401, 2, 310199
    X, _ = bi.mixtures.isotropic_blobs(m, n, 40, seed, box=3.0)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    ctx = bm.bm_create(cfg, dev(X))
    try:
        junk = [torch.full((m, n), 1e3, dtype=torch.float32, device="cuda:0") for _ in range(4)]
        bm.bm_fit_chunk(ctx, T)
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        bm.bm_get_state(ctx, C, mask)
        lab = torch.empty(m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, lab)
        del junk
    finally:
        bm.bm_destroy(ctx)
    A, sse_ref, d1, d2 = o.final_assignment(X, C, mask.astype(bool))
    assert labels_match(host(lab), A, d1, d2)[0] == 0
    assert rel(sse, sse_ref) <= OBJ_REL


def test_random_whole_jobs_match_oracle(bm):
    # seeded sweep of whole jobs (chunks + final assignment) over n, k, m, s,
    # chunk count, precision form and reinitialisation; non-decisive draws are
    # skipped, every decisive one must match the oracle on every output
    rng = np.random.default_rng(2204)
    ran = 0
    while ran < 40:
        n = int(rng.choice([1, 2, 3, 4, 7, 8, 15, 16, 27, 28, 32, 33, 40, 64, 100, 128]))
        k = int(rng.integers(1, 40))
        m = int(rng.integers(max(k, 10), 6000))
        s = int(rng.integers(k, m + 1))
        T = int(rng.integers(1, 4))
        prec = int(rng.choice([0, 1, 2, 3]))
        init = int(rng.choice([0, 0, 0, 1]))
        seed = int(rng.integers(1 << 20))
        comps = int(rng.integers(1, 50))
        box = float(rng.choice([3.0, 8.0, 20.0]))
        X, _ = bi.mixtures.isotropic_blobs(m, n, comps, seed, box=box)
        draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
        st, recs = o.big_means(X, k, draws, init="forgy" if init == 1 else "kmeans++")
        mgs = [_margins(r) for r in recs]
        if not all(g["gap"] >= 1e-5 and g["stop"] >= 1e-6 and g["keep"] >= 1e-6
                   and g["kpp"] >= KPP_BAND and g["pot"] >= 1e-6 for g in mgs):
            continue
        case = dict(m=m, n=n, k=k, s=s, T=T, prec=prec, init=init, seed=seed)
        cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec, init=init)
        ctx = bm.bm_create(cfg, dev(X))
        try:
            rep = bm.bm_fit_chunk(ctx, T)
            C = np.zeros((k, n), np.float32)
            mask = np.zeros(k, np.uint8)
            f_opt, _ = bm.bm_get_state(ctx, C, mask)
            lab = torch.empty(m, dtype=torch.int32, device="cuda:0")
            sse = bm.bm_assign(ctx, lab)
        finally:
            bm.bm_destroy(ctx)
        ran += 1
        assert rep["accepted"] == sum(r.accepted for r in recs), case
        assert rep["lloyd_iters"] == sum(r.iters for r in recs), case
        assert np.array_equal(mask.astype(bool), st.live), case
        assert rel(f_opt, st.f_opt) <= OBJ_REL, case
        assert centroids_close(C, st.C, st.live) <= CEN_REL, case
        A, sse_ref, d1, d2 = o.final_assignment(X, st.C.astype(np.float32), st.live)
        assert labels_match(host(lab), A, d1, d2)[0] == 0, case
        assert rel(sse, sse_ref) <= OBJ_REL, case
