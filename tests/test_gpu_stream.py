"""Streaming contexts (bm_stream_create / bm_stream_push): each pushed portion
is one chunk's sample; against the oracle's chunk on the same rows."""
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


def _portions(n, k, seed, sizes):
    X, _ = bi.mixtures.isotropic_blobs(sum(sizes), n, 2 * k, seed, box=8.0)
    out, a = [], 0
    for r in sizes:
        out.append(X[a:a + r])
        a += r
    return out


@pytest.mark.parametrize("n,k,sizes,seed,init,prec", [
    (6, 8, [3000, 2500, 4000, 3500, 1200], 1, "kmeans++", 0),
    (96, 30, [2000, 1800, 2000], 0, "kmeans++", 3),     # tensor-core kernel
    (28, 12, [5000, 4000, 4500], 1, "forgy", 0),
])
def test_stream_portions_match_oracle(bm, n, k, sizes, seed, init, prec):
    P = _portions(n, k, seed, sizes)
    st = o.BigMeansState(k, n)
    recs = []
    for t, p in enumerate(P):
        recs.append(o.big_means_chunk(p, st, np.arange(len(p)), bi.kpp_uniform_first(seed, t),
                                      bi.kpp_uniforms(seed, t, k), t=t, init=init))
    if init == "kmeans++":
        _assert_decisive(recs)
    code = bm.BM_INIT_FORGY if init == "forgy" else bm.BM_INIT_KMEANSPP
    cfg = bm.bm_config_default(m=1, n=n, k=k, s=max(sizes), seed=seed, precision=prec, init=code)
    stream = torch.cuda.Stream()
    ctx = bm.bm_stream_create(cfg, stream.cuda_stream)
    try:
        accepted = iters = 0
        for p in P:
            rep = bm.bm_stream_push(ctx, dev(p), len(p))
            accepted += rep["accepted"]
            iters += rep["lloyd_iters"]
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt, t = bm.bm_get_state(ctx, C, mask)
        with pytest.raises(bm.BigMeansError):
            bm.bm_fit_chunk(ctx, 1)       # no dataset to sample from
    finally:
        bm.bm_destroy(ctx)
    assert t == len(P)
    assert accepted == sum(r.accepted for r in recs) and iters == sum(r.iters for r in recs)
    assert np.array_equal(mask.astype(bool), st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
