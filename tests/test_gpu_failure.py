"""Failure detection without a GPU fault: a device wait that runs out reports
BM_ETIMEOUT through its status word, and the device stays usable."""
import time

import numpy as np
import pytest

import bminputs as bi
from gpu_helpers import dev, rel, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


def test_barrier_wait_times_out_and_reports(bm):
    t0 = time.time()
    st = bm.bm_selftest_wait_timeout(200)
    dt = time.time() - t0
    assert st == bm.BM_ETIMEOUT
    assert 0.15 < dt < 5.0


def test_device_usable_after_a_timeout(bm):
    assert bm.bm_selftest_wait_timeout(50) == bm.BM_ETIMEOUT
    m, n, k, s = 5000, 6, 4, 1000
    X, _ = bi.mixtures.isotropic_blobs(m, n, k, 3)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=3)
    runs = []
    for _ in range(2):
        stream = torch.cuda.Stream()
        ctx = bm.bm_create(cfg, dev(X), stream.cuda_stream)
        try:
            bm.bm_fit_chunk(ctx, 3)
            runs.append(bm.bm_assign(ctx))
        finally:
            bm.bm_destroy(ctx)
        assert bm.bm_selftest_wait_timeout(20) == bm.BM_ETIMEOUT
    assert runs[0] == runs[1] and np.isfinite(runs[0])
