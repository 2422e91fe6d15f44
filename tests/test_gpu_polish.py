"""Full-data Lloyd polish (bm_polish) against the oracle's Lloyd on all of X,
started from the same incumbent (Big-means run by the oracle, handed over
through bm_set_state)."""
import numpy as np
import pytest

import bminputs as bi
import oracle as o
from gpu_helpers import CEN_REL, OBJ_REL, centroids_close, dev, rel, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


# (name, m, n, k, s, chunks, precision): row-in-register, tiled FP32 and
# tensor-core plans (n = 384, k = 100 has no FP32 tables)
CASES = [("blobs2d", 20000, 2, 10, 2000, 5, 0), ("iso28", 60000, 28, 25, 5000, 4, 0),
         ("iso64", 40000, 64, 33, 4000, 3, 0), ("iso384", 12000, 384, 100, 3000, 2, 0),
         ("iso8", 50000, 8, 16, 5000, 3, 3)]


@pytest.mark.parametrize("name,m,n,k,s,T,prec", CASES)
def test_polish_matches_oracle_lloyd(bm, name, m, n, k, s, T, prec):
    seed = 0
    if name == "blobs2d":
        X = bi.mixtures.blobs_2d(seed)
    else:
        X, _ = bi.mixtures.isotropic_blobs(m, n, 2 * k, seed, box=6.0)
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    st, _ = o.big_means(X, k, draws)
    C0 = st.C.astype(np.float32)
    res = o.lloyd(X, C0.astype(np.float64), st.live.copy())
    assert res.min_gap >= 1e-5 and res.stop_margin >= 1e-6, "not decisive"
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    stream = torch.cuda.Stream()
    ctx = bm.bm_create(cfg, dev(X), stream.cuda_stream)
    try:
        bm.bm_set_state(ctx, C0, st.live.astype(np.uint8), st.f_opt, T)
        f, iters = bm.bm_polish(ctx)
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt, _ = bm.bm_get_state(ctx, C, mask)
        sse = bm.bm_assign(ctx)
    finally:
        bm.bm_destroy(ctx)
    assert iters == res.iters
    assert np.array_equal(mask.astype(bool), res.live)
    assert rel(f, res.f) <= OBJ_REL
    assert centroids_close(C, res.C, res.live) <= CEN_REL
    assert f_opt == st.f_opt                      # the sample objective is kept
    # polishing never raises the full-data objective
    _, sse0, _, _ = o.final_assignment(X, C0, st.live)
    assert sse <= sse0 * (1 + 1e-6)
