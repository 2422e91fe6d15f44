"""The job server (bm_submit): a job's results in a concurrent mix equal the
same job run alone; admission control, waiting, cancellation and counters."""
import threading
import time

import numpy as np
import pytest

import bminputs as bi
from gpu_helpers import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


# (m, n, k, s, precision, chunks): the row-in-register, tiled FP32 and
# tensor-core kernels, FP32 and BF16 forms
MIX = [(20_000, 8, 10, 2_000, 0, 6), (30_000, 28, 25, 5_000, 3, 5),
       (12_000, 68, 40, 3_000, 3, 4), (25_000, 2, 5, 25_000, 0, 3),
       (8_000, 128, 50, 4_000, 0, 3), (15_000, 40, 7, 1_500, 1, 5)]


def _alone(bm, X, cfg, chunks):
    stream = torch.cuda.Stream()
    ctx = bm.bm_create(cfg, X, stream.cuda_stream)
    try:
        rep = bm.bm_fit_chunk(ctx, chunks)
        labels = torch.empty(cfg.m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, labels)
        C = np.zeros((cfg.k, cfg.n), np.float32)
        mask = np.zeros(cfg.k, np.uint8)
        f_opt, _ = bm.bm_get_state(ctx, C, mask)
    finally:
        bm.bm_destroy(ctx)
    return sse, f_opt, rep["lloyd_iters"], C, mask, host(labels)


def test_mix_results_equal_jobs_run_alone(bm):
    data = [dev(bi.mixtures.isotropic_blobs(m, n, max(2 * k, 4), i)[0])
            for i, (m, n, k, s, p, T) in enumerate(MIX)]
    # the server caps a job's CTAs at SMs / workers; run alone with that cap
    cap = -(-torch.cuda.get_device_properties(0).multi_processor_count // 3)
    cfgs = [bm.bm_config_default(m=m, n=n, k=k, s=s, seed=10 + i, precision=p, max_ctas=cap)
            for i, (m, n, k, s, p, T) in enumerate(MIX)]
    sv = bm.bm_server_create(workers=3)
    try:
        outs, tickets = [], []
        for rep in range(2):   # every job twice, all in flight together
            for i, (m, n, k, s, p, T) in enumerate(MIX):
                lab = torch.empty(m, dtype=torch.int32, device="cuda:0")
                C = np.zeros((k, n), np.float32)
                mask = np.zeros(k, np.uint8)
                tickets.append(bm.bm_submit(sv, cfgs[i], data[i], T, lab, C, mask))
                outs.append((i, lab, C, mask))
        results = [bm.bm_wait(sv, t) for t in tickets]
        stats = bm.bm_server_stats(sv)
    finally:
        bm.bm_server_destroy(sv)
    assert stats["submitted"] == stats["completed"] == 2 * len(MIX)
    assert stats["running"] == 0 and stats["queued"] == 0 and stats["memory_in_use"] == 0
    for (i, lab, C, mask), r in zip(outs, results):
        assert r["status"] == 0
        assert r["latency_s"] >= r["run_s"] > 0.0
        sse, f_opt, iters, C1, mask1, lab1 = _alone(bm, data[i], cfgs[i], MIX[i][5])
        assert r["sse"] == sse and r["f_opt"] == f_opt and r["lloyd_iters"] == iters
        assert np.array_equal(C, C1) and np.array_equal(mask, mask1)
        assert np.array_equal(host(lab), lab1)


def test_results_do_not_depend_on_the_worker_count(bm):
    # a job without its own CTA cap runs with the server's job_ctas (default
    # ceil(SMs / 2)) whatever the number of workers: the same bits under
    # servers of 1 and 6 workers, and those of the job alone with that cap
    m, n, k, s, T = 60_000, 28, 12, 8_000, 3
    X = dev(bi.mixtures.isotropic_blobs(m, n, 20, 5)[0])
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=5, precision=1)
    out = []
    for workers in (1, 6):
        sv = bm.bm_server_create(workers=workers)
        try:
            C = np.zeros((k, n), np.float32)
            mask = np.zeros(k, np.uint8)
            lab = torch.empty(m, dtype=torch.int32, device="cuda:0")
            r = bm.bm_wait(sv, bm.bm_submit(sv, cfg, X, T, lab, C, mask))
        finally:
            bm.bm_server_destroy(sv)
        assert r["status"] == 0
        out.append((r["sse"], r["f_opt"], C, mask, host(lab)))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2]) and np.array_equal(out[0][4], out[1][4])
    cap = -(-torch.cuda.get_device_properties(0).multi_processor_count // 2)
    alone_cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=5, precision=1, max_ctas=cap)
    sse, f_opt, _, C1, mask1, lab1 = _alone(bm, X, alone_cfg, T)
    assert out[0][0] == sse and out[0][1] == f_opt and np.array_equal(out[0][2], C1)
    assert np.array_equal(out[0][4], lab1)


def test_admission_wait_cancel_and_callbacks(bm):
    m, n, k, s = 400_000, 28, 25, 50_000
    X = dev(bi.mixtures.isotropic_blobs(m, n, 40, 1)[0])
    slow = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=1)
    small = bm.bm_config_default(m=5_000, n=4, k=3, s=1_000, seed=2)
    sv = bm.bm_server_create(workers=1, max_queue=1, memory_budget=64 << 20)
    seen = {}
    done = threading.Event()

    def cb(ticket, res):
        seen[ticket] = res["status"]
        done.set()

    try:
        # a job larger than the whole budget is refused outright (its
        # sample-plan bitmaps alone take about 256 MB)
        huge = bm.bm_config_default(m=100_000_000, n=8, k=10, s=50_000, seed=3)
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_submit(sv, huge, X, 1)
        assert e.value.status == bm.BM_ENOMEM
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_submit(sv, slow, X, 0)
        assert e.value.status == bm.BM_EINVAL
        t_slow = bm.bm_submit(sv, slow, X, 400)        # occupies the only worker
        t0 = time.time()
        while bm.bm_server_stats(sv)["running"] != 1:   # until the worker has taken it
            assert time.time() - t0 < 10.0
            time.sleep(0.0005)
        t_cb = bm.bm_submit(sv, small, X, 2, callback=cb)   # waits in the queue
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_submit(sv, small, X, 2)              # the queue is full
        assert e.value.status == bm.BM_EBUSY
        assert bm.bm_wait(sv, t_slow, timeout=0.0) is None   # still running
        st = bm.bm_server_stats(sv)
        assert st["rejected_busy"] == 1 and st["rejected_memory"] == 1
    finally:
        bm.bm_server_destroy(sv)   # the slow job finishes, the queued one is cancelled
    assert done.wait(5.0)
    assert seen == {t_cb: bm.BM_ECANCELLED}


def test_callbacks_report_completed_jobs(bm):
    X = dev(bi.mixtures.isotropic_blobs(20_000, 6, 8, 5)[0])
    cfg = bm.bm_config_default(m=20_000, n=6, k=8, s=2_000, seed=5)
    got = []
    lock = threading.Lock()
    all_done = threading.Event()

    def cb(ticket, res):
        with lock:
            got.append((ticket, res["status"], res["sse"]))
            if len(got) == 5:
                all_done.set()

    sv = bm.bm_server_create(workers=2)
    try:
        tickets = [bm.bm_submit(sv, cfg, X, 3, callback=cb) for _ in range(5)]
        assert all_done.wait(30.0)
    finally:
        bm.bm_server_destroy(sv)
    assert sorted(t for t, _, _ in got) == sorted(tickets)
    assert all(st == 0 for _, st, _ in got)
    assert len({sse for _, _, sse in got}) == 1   # same job, same result


@pytest.mark.parametrize("m,n,k,s,seed,T,prec,cap", [
    (3000, 64, 33, 1000, 0, 3, 3, 3),     # tensor-core chunk kernel on 3 SMs
    (20000, 2, 10, 2000, 0, 4, 0, 5),     # row-in-register kernel on 5 SMs
])
def test_capped_jobs_match_the_oracle(bm, m, n, k, s, seed, T, prec, cap):
    import oracle as o
    from gpu_helpers import CEN_REL, OBJ_REL, centroids_close, rel
    from test_gpu_parity import _assert_decisive
    if n == 2:
        X = bi.mixtures.blobs_2d(seed)
    else:
        X, _ = bi.mixtures.isotropic_blobs(m, n, max(k, 2), seed, box=8.0)
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    st, recs = o.big_means(X, k, draws)
    _assert_decisive(recs)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec, max_ctas=cap)
    sse, f_opt, iters, C, mask, lab = _alone(bm, dev(X), cfg, T)
    assert iters == sum(r.iters for r in recs)
    assert np.array_equal(mask.astype(bool), st.live)
    assert rel(f_opt, st.f_opt) <= OBJ_REL
    assert centroids_close(C, st.C, st.live) <= CEN_REL
