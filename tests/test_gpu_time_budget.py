"""The paper's stop condition: Big-means runs chunks until a time budget has
elapsed (Sec. 5, the experiments' only stop rule).  bm_fit_chunk(ctx, 0)
with cfg.time_budget_s does that; the run it makes is an ordinary run of
that many chunks, so replaying the same number of chunks from scratch must
give the same incumbent bit for bit, and its first chunks must match the
FP64 oracle."""
import numpy as np
import pytest

import bminputs as bi
import oracle as o
from gpu_helpers import CEN_REL, OBJ_REL, centroids_close, dev, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


def _state(bm, ctx, k, n):
    C = np.zeros((k, n), np.float32)
    mask = np.zeros(k, np.uint8)
    f_opt, t = bm.bm_get_state(ctx, C, mask)
    return C, mask, f_opt, t


@pytest.mark.parametrize("budget", [0.02, 0.2])
def test_time_budget_runs_until_it_elapses(bm, budget):
    m, n, k, s, seed = 20_000, 2, 10, 2_000, 0
    X = bi.mixtures.blobs_2d(seed)
    Xd = dev(X)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, time_budget_s=budget)
    ctx = bm.bm_create(cfg, Xd)
    try:
        rep = bm.bm_fit_chunk(ctx, 0)
        C, mask, f_opt, t = _state(bm, ctx, k, n)
    finally:
        bm.bm_destroy(ctx)
    T = rep["chunks"]
    assert T >= 2 and t == T
    assert budget <= rep["seconds"] < budget + 1.0
    # the same number of chunks, by count: the same incumbent, bit for bit
    cfg2 = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed)
    ctx2 = bm.bm_create(cfg2, Xd)
    try:
        rep2 = bm.bm_fit_chunk(ctx2, T)
        C2, mask2, f2, t2 = _state(bm, ctx2, k, n)
    finally:
        bm.bm_destroy(ctx2)
    assert rep2["accepted"] == rep["accepted"] and rep2["lloyd_iters"] == rep["lloyd_iters"]
    assert np.array_equal(C, C2) and np.array_equal(mask, mask2) and f_opt == f2 and t2 == t
    # and the run is Alg. 1: its first chunks against the oracle
    Tc = min(T, 20)
    ctx3 = bm.bm_create(cfg2, Xd)
    try:
        bm.bm_fit_chunk(ctx3, Tc)
        C3, mask3, f3, _ = _state(bm, ctx3, k, n)
    finally:
        bm.bm_destroy(ctx3)
    st, _ = o.big_means(X, k, [bi.chunk_draws(seed, q, m, s, k) for q in range(Tc)])
    assert np.array_equal(mask3.astype(bool), st.live)
    assert rel(f3, st.f_opt) <= OBJ_REL and centroids_close(C3, st.C, st.live) <= CEN_REL


def test_zero_chunks_without_a_budget_is_invalid(bm):
    X = bi.mixtures.blobs_2d(0)
    cfg = bm.bm_config_default(m=20_000, n=2, k=10, s=2_000, seed=0)
    ctx = bm.bm_create(cfg, dev(X))
    try:
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_fit_chunk(ctx, 0)
        assert e.value.status == bm.BM_EINVAL
    finally:
        bm.bm_destroy(ctx)
