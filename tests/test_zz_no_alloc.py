"""bm_assign_rows_noalloc against bm_assign_rows, through the C ABI.

The allocation-free entry point exists for callers that cannot allocate
device memory when they need an assignment (memory handed to their own pool
allocator, or a loop where cudaMalloc's device-wide synchronisation is not
acceptable).  It must give the same labels and per-row distances as the
allocating entry point and the same SSE within the parity tolerance, on two
calls in a row -- the second call reuses the scratch array the first one
left behind.  This file is named to be collected last.
"""
import numpy as np
import pytest

import bminputs as bi
from gpu_helpers import OBJ_REL, dev, host, rel, require_gpu, torch

pytestmark = pytest.mark.gpu


def _case(m, n, k, seed):
    X, _ = bi.mixtures.isotropic_blobs(m, n, k, seed, box=5.0)
    rng = np.random.default_rng(seed)
    C = (X[rng.choice(m, k, replace=False)]
         + rng.normal(scale=0.2, size=(k, n))).astype(np.float32)
    live = np.ones(k, np.uint8)
    live[rng.choice(k, k // 5, replace=False)] = 0
    return X, C, live


def test_noalloc_assign_matches_allocating_entry_point_on_consecutive_calls():
    require_gpu()
    import paper_2204_07485_gb300 as bm
    # two calls in a row: the row-in-register kernel, then the tiled kernel
    for m, n, k, seed in [(200_003, 28, 25, 0), (50_001, 96, 40, 1)]:
        X, C, live = _case(m, n, k, seed)
        Xd, Cd, md = dev(X), dev(C), dev(live)
        lab_ref = torch.empty(m, dtype=torch.int32, device="cuda:0")
        dmin_ref = torch.empty(m, dtype=torch.float32, device="cuda:0")
        sse_ref = bm.bm_assign_rows(Xd, m, n, Cd, md, k, lab_ref, dmin_ref)
        lab = torch.full((m,), -1, dtype=torch.int32, device="cuda:0")
        dmin = torch.full((m,), -1.0, dtype=torch.float32, device="cuda:0")
        sse = bm.bm_assign_rows_noalloc(Xd, m, n, Cd, md, k, lab, dmin)
        assert torch.equal(lab, lab_ref)
        np.testing.assert_allclose(host(dmin), host(dmin_ref),
                                   rtol=(n + 2) * 2.0 ** -24, atol=0)
        assert rel(sse, sse_ref) <= OBJ_REL


def test_noalloc_rejects_bad_arguments():
    require_gpu()
    import paper_2204_07485_gb300 as bm
    X, C, live = _case(1000, 4, 5, 2)
    with pytest.raises(bm.BigMeansError) as e:
        bm.bm_assign_rows_noalloc(dev(X), 1000, 4, dev(C), dev(np.zeros(5, np.uint8)), 5)
    assert e.value.status == bm.BM_EINVAL
    C200 = np.zeros((200, 4), np.float32)
    with pytest.raises(bm.BigMeansError) as e:
        bm.bm_assign_rows_noalloc(dev(X), 1000, 4, dev(C200), dev(np.ones(200, np.uint8)), 200)
    assert e.value.status == bm.BM_EUNSUPPORTED
