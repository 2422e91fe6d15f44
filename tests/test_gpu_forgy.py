"""Forgy reinitialisation (BM_INIT_FORGY) against the oracle on decisive
whole runs of the three chunk-kernel families."""
import numpy as np
import pytest

import bminputs as bi
import oracle as o
from gpu_helpers import CEN_REL, OBJ_REL, centroids_close, dev, rel, require_gpu, torch
from test_gpu_parity import _assert_decisive

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


@pytest.mark.parametrize("m,n,k,s,T,seed,prec", [
    (20000, 2, 10, 2000, 6, 2, 0),      # row-in-register kernel
    (30000, 28, 25, 6000, 5, 0, 0),
    (8000, 64, 20, 2000, 4, 0, 0),      # tiled FP32 kernel
    (3000, 384, 50, 1500, 3, 2, 3),     # tensor-core kernel
])
def test_forgy_runs_match_oracle(bm, m, n, k, s, T, seed, prec):
    X, _ = bi.mixtures.isotropic_blobs(m, n, 2 * k, seed, box=8.0)
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    st, recs = o.big_means(X, k, draws, init="forgy")
    _assert_decisive(recs)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec,
                               init=bm.BM_INIT_FORGY)
    stream = torch.cuda.Stream()
    ctx = bm.bm_create(cfg, dev(X), stream.cuda_stream)
    try:
        rep = bm.bm_fit_chunk(ctx, T)
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt, _ = bm.bm_get_state(ctx, C, mask)
    finally:
        bm.bm_destroy(ctx)
    assert rep["accepted"] == sum(r.accepted for r in recs)
    assert rep["lloyd_iters"] == sum(r.iters for r in recs)
    assert rep["n_d"] == sum(r.n_d for r in recs)
    assert np.array_equal(mask.astype(bool), st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
