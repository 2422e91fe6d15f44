"""CUDA-graph replay of bm_fit_chunk: a recorded launch sequence, replayed,
gives bit-for-bit the results of launching the kernels one at a time."""
import numpy as np
import pytest

import bminputs as bi
from gpu_helpers import dev, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


def _jobs(bm, X, cfg, plan):
    """Runs `plan` (a list of bm_fit_chunk chunk counts, None = bm_reset) on a
    private stream; returns the state after every fit."""
    stream = torch.cuda.Stream()
    ctx = bm.bm_create(cfg, dev(X), stream.cuda_stream)
    out = []
    try:
        for step in plan:
            if step is None:
                bm.bm_reset(ctx)
                continue
            rep = bm.bm_fit_chunk(ctx, step)
            C = np.zeros((cfg.k, cfg.n), np.float32)
            mask = np.zeros(cfg.k, np.uint8)
            f_opt, t = bm.bm_get_state(ctx, C, mask)
            out.append((rep["accepted"], rep["lloyd_iters"], f_opt, t, C, mask))
    finally:
        bm.bm_destroy(ctx)
    return out


@pytest.mark.parametrize("m,n,k,s,prec", [(30000, 12, 16, 3000, 0), (20000, 96, 40, 6000, 3),
                                          (20000, 2, 10, 2000, 0)])
def test_graph_replay_matches_direct_launches(bm, m, n, k, s, prec):
    X, _ = bi.mixtures.isotropic_blobs(m, n, 2 * k, 4)
    # the same job three times (record once, replay twice), then a fit split
    # into pieces that start from other launch states, then 70 chunks (a
    # second sample-plan window)
    plan = [None, 7, None, 7, None, 7, None, 3, 4, 5, None, 70]
    runs = []
    for graphs in (0, 1):
        cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=42, precision=prec, graphs=graphs)
        runs.append(_jobs(bm, X, cfg, plan))
    for a, b in zip(*runs):
        assert a[:4] == b[:4]
        assert np.array_equal(a[4], b[4]) and np.array_equal(a[5], b[5])
    # the three identical jobs agree with each other
    assert all(runs[1][i][2] == runs[1][0][2] for i in range(3))


def test_default_stream_falls_back_to_direct_launches(bm):
    m, n, k, s = 5000, 3, 4, 500
    X, _ = bi.mixtures.isotropic_blobs(m, n, k, 1)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=1)
    ctx = bm.bm_create(cfg, dev(X))   # legacy default stream: nothing to record on
    try:
        rep = bm.bm_fit_chunk(ctx, 4)
    finally:
        bm.bm_destroy(ctx)
    assert rep["chunks"] == 4
