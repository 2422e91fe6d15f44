"""Repeated K-means++ reseeds (Sec. 3.3; three candidates, Sec. 5) on the
three chunk-kernel families, with the exchange self-check on.

The CTAs of a chunk launch hand each other their D^2 block sums, the
candidate rows and the candidates' potentials between grid barriers.  Each
value carries a tag of its launch and slot, and a reader that finds the tag
not yet written waits for it and counts a late read (bm_sync_late_reads).
These tests repeat the step-level reseed and whole first chunks (every
centroid reseeded, then Lloyd) many times: every repeat must equal the FP64
oracle (decisive cases: no inverse-CDF target within 5e-8 * sum(D^2) of a
prefix boundary, no two candidate potentials within 1e-6), equal the first
repeat bit for bit, and leave the late-read count unchanged.

BM_KPP_REPEAT sets the repeats (default 3; a dedicated run uses hundreds).
"""
import math
import os

import numpy as np
import pytest

import bminputs as bi
import oracle as o
from gpu_helpers import CEN_REL, OBJ_REL, centroids_close, dev, host, rel, require_gpu

pytestmark = pytest.mark.gpu

REPEAT = int(os.environ.get("BM_KPP_REPEAT", "3"))
KPP_BAND = 5e-8


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


def _assert_picks_decisive(picks):
    for p in picks:
        assert p.boundary_margin >= KPP_BAND, "not decisive: %r" % p.boundary_margin
        pots = sorted(set(p.potentials))
        assert len(pots) < 2 or (pots[1] - pots[0]) / pots[0] >= 1e-6


STEP_CASES = [  # (m, n, k, s, seed): all slots degenerate, chunk 0
    (8000, 28, 25, 5000, 1),      # row-in-register kernel
    (6000, 128, 50, 3000, 2),     # tiled FP32 kernel, 12 CTAs
    (6000, 384, 100, 3000, 0),    # tensor-core kernel (FP32 tables beyond shared memory)
]


@pytest.mark.parametrize("m,n,k,s,seed", STEP_CASES)
def test_step_reseed_repeated(bm, m, n, k, s, seed):
    X, _ = bi.mixtures.isotropic_blobs(m, n, max(k, 2), seed)
    idx, uf, u = bi.chunk_draws(seed, 0, m, s, k)
    P = X[idx]
    picks = []
    C0 = np.zeros((k, n), np.float32)
    live0 = np.zeros(k, bool)
    C_ref, live_ref = o.kmeanspp_reseed(P, C0, live0, uf, u, 3, picks)
    _assert_picks_decisive(picks)
    Pd = dev(P)
    late0 = bm.bm_sync_late_reads()
    for r in range(REPEAT):
        Cd, md = dev(C0), dev(live0.astype(np.uint8))
        bm.bm_kpp_reseed(Pd, s, n, k, Cd, md, seed, 0, 3)
        assert np.array_equal(host(md).astype(bool), live_ref), "repeat %d" % r
        assert np.array_equal(host(Cd).astype(np.float64), C_ref), "repeat %d" % r
    assert bm.bm_sync_late_reads() == late0


CHUNK_CASES = [  # (m, n, k, s, seed, precision)
    (20000, 28, 25, 5000, 0, 0),     # row-in-register kernel
    (12000, 128, 50, 6000, 0, 0),    # tiled FP32 kernel
    (12000, 128, 50, 6000, 0, 3),    # tensor-core kernel (split BF16 + exact rescoring)
]


@pytest.mark.parametrize("m,n,k,s,seed,prec", CHUNK_CASES)
def test_first_chunk_repeated(bm, m, n, k, s, seed, prec):
    X, _ = bi.mixtures.isotropic_blobs(m, n, max(k, 2), seed)
    draws = [bi.chunk_draws(seed, 0, m, s, k)]
    st, recs = o.big_means(X, k, draws)
    rec = recs[0]
    _assert_picks_decisive(rec.picks)
    assert rec.lloyd.min_gap >= 1e-5 and rec.lloyd.stop_margin >= 1e-6
    Xd = dev(X)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    ctx = bm.bm_create(cfg, Xd)
    late0 = bm.bm_sync_late_reads()
    first = None
    try:
        for r in range(REPEAT):
            bm.bm_reset(ctx)
            rep = bm.bm_fit_chunk(ctx, 1)
            C = np.zeros((k, n), np.float32)
            mask = np.zeros(k, np.uint8)
            f_opt = bm.bm_objective(ctx, C, mask)
            if first is None:
                first = (C.copy(), mask.copy(), f_opt)
                assert rep["lloyd_iters"] == rec.iters
                assert np.array_equal(mask.astype(bool), st.live)
                assert rel(f_opt, st.f_opt) <= OBJ_REL
                assert centroids_close(C, st.C, st.live) <= CEN_REL
            else:
                assert np.array_equal(C, first[0]) and np.array_equal(mask, first[1]), \
                    "repeat %d differs" % r
                assert f_opt == first[2], "repeat %d" % r
    finally:
        bm.bm_destroy(ctx)
    assert bm.bm_sync_late_reads() == late0
    assert math.isfinite(first[2])
