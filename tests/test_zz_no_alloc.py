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
        # the same kernel and grid as the allocating call: equal bit for bit
        assert torch.equal(lab, lab_ref)
        assert torch.equal(dmin, dmin_ref)
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


def test_noalloc_sse_only_call_matches():
    """labels and dmin both NULL: only the objective is produced."""
    require_gpu()
    import paper_2204_07485_gb300 as bm
    m, n, k = 30_011, 12, 17
    X, C, live = _case(m, n, k, 3)
    Xd, Cd, md = dev(X), dev(C), dev(live)
    sse_ref = bm.bm_assign_rows(Xd, m, n, Cd, md, k)
    for _ in range(2):
        sse = bm.bm_assign_rows_noalloc(Xd, m, n, Cd, md, k)
        assert rel(sse, sse_ref) <= OBJ_REL


def test_noalloc_refuses_tables_beyond_shared_memory():
    """n = 384, k = 100: the FP32 centroid table does not fit in shared
    memory.  bm_assign_rows switches to the tensor-core kernel (whose scratch
    grows with m); the allocation-free call refuses the shape instead."""
    require_gpu()
    import paper_2204_07485_gb300 as bm
    m, n, k = 4_000, 384, 100
    X, C, live = _case(m, n, k, 4)
    Xd, Cd, md = dev(X), dev(C), dev(live)
    lab_ref = torch.empty(m, dtype=torch.int32, device="cuda:0")
    bm.bm_assign_rows(Xd, m, n, Cd, md, k, lab_ref)
    with pytest.raises(bm.BigMeansError) as e:
        bm.bm_assign_rows_noalloc(Xd, m, n, Cd, md, k)
    assert e.value.status == bm.BM_EUNSUPPORTED
