"""GPU parity of the tensor-core chunk kernel (rows wider than 32 features).

A context created with a BF16, split-BF16 or E4M3 precision form runs every
Lloyd and K-means++ assignment of a chunk on the tensor cores with exact
FP32 rescoring; an FP32 context whose shared-memory tables do not fit takes
the same kernel.  Cases
are decisive in the sense of test_gpu_parity (asserted from the oracle's own
record), so the GPU must reach the oracle's decisions: labels, degenerate
sets, Lloyd iteration counts, keep-the-best outcomes, and objectives and
centroids within 1e-6 relative.
"""
import numpy as np
import pytest

import bminputs as bi
import oracle as o
from gpu_helpers import (CEN_REL, OBJ_REL, centroids_close, dev, host, labels_match, rel,
                         require_gpu, torch)
from test_gpu_parity import _assert_decisive

pytestmark = pytest.mark.gpu
BF16, FP8, BF16X3 = 1, 2, 3


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


def _run(bm, X, cfg, T):
    ctx = bm.bm_create(cfg, dev(X))
    try:
        rep = bm.bm_fit_chunk(ctx, T)
        C = np.zeros((cfg.k, cfg.n), np.float32)
        mask = np.zeros(cfg.k, np.uint8)
        f_opt, _ = bm.bm_get_state(ctx, C, mask)
        labels = torch.empty(cfg.m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, labels)
    finally:
        bm.bm_destroy(ctx)
    return rep, C, mask.astype(bool), f_opt, host(labels), sse


@pytest.mark.parametrize("m,n,k,s,seed,T,prec", [
    (1200, 40, 1, 400, 0, 3, BF16X3),       # k = 1
    (3000, 64, 33, 1000, 0, 3, BF16X3),     # k just above one 32-column group
    (4000, 128, 50, 2000, 1, 3, BF16X3),
    (2500, 200, 17, 1300, 0, 3, BF16X3),    # n not a multiple of 64 (K padding)
    (1000, 33, 7, 999, 0, 2, BF16X3),       # n = 33: one padded block, s ~ m
    (5000, 68, 100, 2500, 0, 2, BF16X3),
    (3000, 384, 100, 1500, 0, 2, BF16X3),   # six K blocks, n16 = 112
    (3000, 384, 100, 1500, 0, 2, 0),        # FP32 form: tables too large, same kernel
    # BF16 screening (one plane, one MMA per product; looser bound, more rescoring)
    (4000, 128, 50, 2000, 1, 3, BF16),
    (2500, 200, 17, 1300, 0, 3, BF16),
    (1000, 33, 7, 999, 0, 2, BF16),
    (3000, 384, 100, 1500, 0, 2, BF16),
    (1200, 40, 1, 400, 0, 3, BF16),
    # E4M3 screening (K blocks of 128 features, per-row and per-chunk scales)
    (3000, 384, 100, 1500, 0, 2, FP8),      # three K blocks, n16 = 112
    (4000, 128, 50, 2000, 1, 3, FP8),
    (2500, 200, 17, 1300, 0, 3, FP8),       # n = 200: second K block padded
    (1000, 33, 7, 999, 0, 2, FP8),
    (5000, 68, 100, 2500, 0, 2, FP8),
    (3000, 64, 33, 1000, 0, 3, FP8),
    (1200, 40, 1, 400, 0, 3, FP8),
])
def test_tc_chunks_match_oracle(bm, m, n, k, s, seed, T, prec):
    X, _ = bi.mixtures.isotropic_blobs(m, n, max(k, 2), seed, box=8.0)
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    st, recs = o.big_means(X, k, draws)
    _assert_decisive(recs)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    rep, C, mask, f_opt, labels, sse = _run(bm, X, cfg, T)
    assert rep["accepted"] == sum(r.accepted for r in recs)
    assert rep["lloyd_iters"] == sum(r.iters for r in recs)
    assert rep["n_d"] == sum(r.n_d for r in recs)
    assert np.array_equal(mask, st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
    A, sse_ref, d1, d2 = o.final_assignment(X, st.C.astype(np.float32), st.live)
    bad, _ = labels_match(labels, A, d1, d2)
    assert bad == 0
    assert rel(sse, sse_ref) <= OBJ_REL


@pytest.mark.parametrize("seed,chunks,prec", [(2, (1, 2, 3, 4, 5), BF16X3),
                                              (2, (1, 2, 3, 4, 5), BF16),
                                              (2, (1, 2, 3, 4, 5), FP8)])
def test_tc_full_size_chunks_teacher_forced(bm, seed, chunks, prec):
    """m = 200,000, n = 128, k = 50, s = 50,000 (a 100-component mixture with
    Dirichlet(0.5) weights): every chunk starts from the oracle's incumbent
    and must end at the oracle's."""
    m, n, k, s = 200_000, 128, 50, 50_000
    X, _ = bi.mixtures.isotropic_blobs(m, n, 100, 0, alpha=0.5)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    ctx = bm.bm_create(cfg, dev(X))
    st = o.BigMeansState(k, n)
    try:
        for t in range(max(chunks) + 1):
            before = st.copy()
            idx, uf, u = bi.chunk_draws(seed, t, m, s, k)
            rec = o.big_means_chunk(X, st, idx, uf, u, t=t)
            if t not in chunks:
                continue
            _assert_decisive([rec])
            bm.bm_set_state(ctx, before.C.astype(np.float32), before.live.astype(np.uint8),
                            before.f_opt, t)
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
    finally:
        bm.bm_destroy(ctx)


def test_tc_and_fp32_kernels_agree(bm):
    # the same job through the tiled FP32 kernel and the tensor-core kernel
    m, n, k, s, T, seed = 3000, 64, 33, 1000, 3, 0
    X, _ = bi.mixtures.isotropic_blobs(m, n, k, seed, box=8.0)
    out = []
    for prec in (0, BF16X3, BF16, FP8):
        cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
        out.append(_run(bm, X, cfg, T))
    r0, C0, m0, f0, l0, s0 = out[0]
    for r1, C1, m1, f1, l1, s1 in out[1:]:
        assert r0["lloyd_iters"] == r1["lloyd_iters"] and r0["accepted"] == r1["accepted"]
        assert np.array_equal(m0, m1)
        assert rel(f0, f1) <= OBJ_REL
        assert centroids_close(C1, C0.astype(np.float64), m0) <= CEN_REL


@pytest.mark.parametrize("prec", [BF16X3, FP8])
def test_tc_runs_are_bitwise_deterministic(bm, prec):
    m, n, k, s, T, seed = 20_000, 96, 40, 6000, 4, 5
    X, _ = bi.mixtures.isotropic_blobs(m, n, 60, seed)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    a = _run(bm, X, cfg, T)
    b = _run(bm, X, cfg, T)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert a[3] == b[3] and np.array_equal(a[4], b[4]) and a[5] == b[5]


def test_tc_op_level_lloyd_for_wide_tables(bm):
    # bm_lloyd with tables too large for the FP32 kernel runs on the tensor cores
    m, n, k, s, seed = 4000, 384, 100, 1500, 0
    X, _ = bi.mixtures.isotropic_blobs(m, n, 2 * k, seed, box=6.0)
    idx, uf, u = bi.chunk_draws(seed, 0, m, s, k)
    P = X[idx]
    C0, live0 = o.kmeanspp_reseed(P, np.zeros((k, n)), np.zeros(k, bool), uf, u)
    res = o.lloyd(P, C0, live0)
    assert res.min_gap >= 1e-5 and res.stop_margin >= 1e-6
    Cd = dev(C0.astype(np.float32))
    md = dev(live0.astype(np.uint8))
    f, iters = bm.bm_lloyd(dev(P), s, n, k, Cd, md)
    assert iters == res.iters
    assert np.array_equal(host(md).astype(bool), res.live)
    assert rel(f, res.f) <= OBJ_REL
    assert centroids_close(host(Cd), res.C, res.live) <= CEN_REL


@pytest.mark.parametrize("prec", [FP8, BF16])
def test_tc_far_incumbent_centroid(bm, prec):
    """A chunk whose incumbent holds a centroid 40 times farther out than the
    largest data value (the E4M3 centroid scale of the chunk then comes from
    that centroid, so the other centroids sit far down the E4M3 range): the
    far centroid loses every member and becomes degenerate, and the chunk
    (accepted: the incumbent objective is +inf) must end at the oracle's
    outcome."""
    m, n, k, s, seed = 6000, 128, 20, 3000, 3
    X, _ = bi.mixtures.isotropic_blobs(m, n, 30, seed, box=8.0)
    st = o.BigMeansState(k, n)
    idx, uf, u = bi.chunk_draws(seed, 0, m, s, k)
    o.big_means_chunk(X, st, idx, uf, u, t=0)
    st.C[3] = 40.0 * np.abs(X).max() * np.where(np.arange(n) % 2 == 1, 1.0, -1.0)
    st.f_opt = np.inf
    before = st.copy()
    idx, uf, u = bi.chunk_draws(seed, 1, m, s, k)
    rec = o.big_means_chunk(X, st, idx, uf, u, t=1)
    _assert_decisive([rec])
    assert rec.accepted and not st.live[3]
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    ctx = bm.bm_create(cfg, dev(X))
    try:
        bm.bm_set_state(ctx, before.C.astype(np.float32), before.live.astype(np.uint8),
                        before.f_opt, 1)
        rep = bm.bm_fit_chunk(ctx, 1)
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt, tc = bm.bm_get_state(ctx, C, mask)
    finally:
        bm.bm_destroy(ctx)
    assert tc == 2
    assert rep["accepted"] == 1 and rep["lloyd_iters"] == rec.iters
    assert np.array_equal(mask.astype(bool), st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
