"""The paper's parallel modes (bm_fit_workers) against the oracle's
sequential simulation of the same rounds.  Cases are decisive for every
worker chunk, and the between-worker choices (the best of a collective round,
the best worker of a competitive run) have a relative margin of at least
1e-6."""
import math

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


def _choice_margin(recs, workers, rounds, mode):
    """Smallest relative gap between the winner and the runner-up of every
    between-worker choice the oracle made."""
    gaps = []
    if mode == "collective":
        for r in range(rounds):
            fs = sorted(rec.f_chunk for rec in recs[r * workers:(r + 1) * workers] if rec.accepted)
            if len(fs) > 1:
                gaps.append((fs[1] - fs[0]) / fs[0])
    else:
        final = []
        for w in range(workers):
            f = math.inf
            for r in range(rounds):
                rec = recs[r * workers + w]
                if rec.accepted:
                    f = rec.f_chunk
            final.append(f)
        fs = sorted(final)
        if len(fs) > 1 and math.isfinite(fs[1]):
            gaps.append((fs[1] - fs[0]) / fs[0])
    return min(gaps or [math.inf])


@pytest.mark.parametrize("mode", ["competitive", "collective"])
@pytest.mark.parametrize("m,n,k,s,W,R,seed,prec", [
    (20000, 2, 10, 2000, 4, 4, 4, 0),
    (30000, 12, 16, 3000, 3, 4, 0, 0),
    (8000, 64, 20, 2000, 3, 3, 2, 3),      # tensor-core chunk kernel
])
def test_workers_match_oracle(bm, m, n, k, s, W, R, seed, prec, mode):
    X, _ = bi.mixtures.isotropic_blobs(m, n, 2 * k, seed, box=8.0)
    draws_of = lambda t: bi.chunk_draws(seed, t, m, s, k)
    st, recs = o.big_means_workers(X, k, draws_of, W, R, mode)
    _assert_decisive(recs)
    assert _choice_margin(recs, W, R, mode) >= 1e-6
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec)
    stream = torch.cuda.Stream()
    ctx = bm.bm_create(cfg, dev(X), stream.cuda_stream)
    code = bm.BM_WORKERS_COLLECTIVE if mode == "collective" else bm.BM_WORKERS_COMPETITIVE
    try:
        rep = bm.bm_fit_workers(ctx, W, R, code)
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt, t = bm.bm_get_state(ctx, C, mask)
    finally:
        bm.bm_destroy(ctx)
    assert t == W * R and rep["chunks"] == W * R
    assert rep["accepted"] == sum(r.accepted for r in recs)
    assert rep["lloyd_iters"] == sum(r.iters for r in recs)
    assert np.array_equal(mask.astype(bool), st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
