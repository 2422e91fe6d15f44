"""Whole free-running GPU runs against the FP64 oracle with decision
following (the oracle's reading R17, tests/parity_follow.py), on the real
draws of the benchmark workloads:

  * m = 20,000, n = 2, k = 10, s = 2,000, seed 0, all 20 chunks;
  * m = 1e6, n = 28, k = 25, s = 50,000, seed 0, all 100 chunks (FP32);
  * m = 1e7, n = 128, k = 50, s = 50,000, seed 0: all 100 chunks of the
    timed job in its timed form (BF16 + exact rescoring; fewer with
    BM_FOLLOW_C3_CHUNKS), then the final assignment of all 1e7 rows against
    the oracle's over every row;
  * m = 2e6, n = 384, k = 100, s = 50,000, seed 0 (per-feature scales
    log-uniform in [0.1, 10]) in the E4M3 form: the first 10 chunks (more or
    fewer with BM_FOLLOW_FP8_CHUNKS), then the final assignment of all 2e6
    rows.

The GPU runs alone: each chunk is one bm_fit_chunk call, and only its
outcome is read.  After every chunk the oracle must reproduce that outcome,
taking the other side of an exempt decision only where needed; the count of
such followed decisions is reported (BM_FOLLOW_REPORT names a JSON-lines
file to append it to) and bounded.
"""
import json
import os
import tempfile

import numpy as np
import pytest

import bminputs as bi
import oracle as o
import parity_follow as pf
from gpu_helpers import OBJ_REL, dev, host, labels_match, rel, require_gpu, torch

pytestmark = pytest.mark.gpu

C3_CHUNKS = int(os.environ.get("BM_FOLLOW_C3_CHUNKS", "100"))
FP8_CHUNKS = int(os.environ.get("BM_FOLLOW_FP8_CHUNKS", "10"))


@pytest.fixture(scope="module")
def bm():
    require_gpu()
    import paper_2204_07485_gb300 as lib
    return lib


def _report(name, **kw):
    path = os.environ.get("BM_FOLLOW_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(case=name, **kw)) + "\n")


def _observer(bm, ctx, k, n):
    def observe(t):
        rep = bm.bm_fit_chunk(ctx, 1)
        C = np.zeros((k, n), np.float32)
        mask = np.zeros(k, np.uint8)
        f_opt, tc = bm.bm_get_state(ctx, C, mask)
        assert tc == t + 1
        return {"accepted": rep["accepted"], "iters": rep["lloyd_iters"], "f_opt": f_opt,
                "C": C, "live": mask.astype(bool)}
    return observe


def _follow(bm, X_host, Xd, m, n, k, s, T, seed, prec=0, Xo=None, draws=None):
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=prec, graphs=0)
    ctx = bm.bm_create(cfg, Xd)
    try:
        draws = draws or [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
        st, recs, followed, bad = pf.follow_run(X_host if Xo is None else Xo, k, draws,
                                                _observer(bm, ctx, k, n))
        return ctx, st, recs, followed, bad
    except Exception:
        bm.bm_destroy(ctx)
        raise


def test_c1_blobs_2d_seed0_free_running(bm):
    m, n, k, s, T, seed = 20_000, 2, 10, 2_000, 20, 0
    X = bi.mixtures.blobs_2d(seed)
    ctx, st, recs, followed, bad = _follow(bm, X, dev(X), m, n, k, s, T, seed)
    try:
        assert bad is None, "chunk %r: no admissible oracle outcome matches" % bad
        labels = torch.empty(m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, labels)
    finally:
        bm.bm_destroy(ctx)
    A, sse_ref, d1, d2 = o.final_assignment(X, st.C, st.live)
    nbad, _ = labels_match(host(labels), A, d1, d2)
    assert nbad == 0 and rel(sse, sse_ref) <= OBJ_REL
    _report("c1_blobs_2d_seed0_T20", followed=[list(f) for f in followed], chunks=T)
    assert len(followed) <= 2


def test_c2_hepmass_like_seed0_all_chunks_free_running(bm):
    m, n, k, s, T, seed = 1_000_000, 28, 25, 50_000, 100, 0
    X = bi.mixtures.hepmass_like(seed, m=m)
    ctx, st, recs, followed, bad = _follow(bm, X, dev(X), m, n, k, s, T, seed)
    try:
        assert bad is None, "chunk %r: no admissible oracle outcome matches" % bad
        labels = torch.empty(m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, labels)
    finally:
        bm.bm_destroy(ctx)
    A, sse_ref, d1, d2 = o.final_assignment(X, st.C, st.live)
    nbad, nties = labels_match(host(labels), A, d1, d2)
    assert nbad == 0 and rel(sse, sse_ref) <= OBJ_REL
    _report("c2_hepmass_like_seed0_T100", followed=[list(f) for f in followed], chunks=T,
            accepted=sum(r.accepted for r in recs), lloyd_iters=sum(r.iters for r in recs),
            final_tie_rows=nties, sse_rel=rel(sse, sse_ref))
    assert len(followed) <= 10


def _follow_device_workload(bm, Xd, m, n, k, s, T, seed, prec, name, max_followed):
    """Free-running chunks of a device-generated workload against the
    oracle (which reads only the chunk rows: a compact copy with remapped
    draws), then the final assignment of all m rows from the oracle's
    incumbent (equal to the GPU's within the parity tolerance) against the
    oracle's over every row."""
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(T)]
    allidx = np.concatenate([np.asarray(d[0], np.int64) for d in draws])
    Xs = Xd[torch.from_numpy(allidx).to("cuda:0")].cpu().numpy()
    cdraws = [(np.arange(q * s, (q + 1) * s), d[1], d[2]) for q, d in enumerate(draws)]
    ctx, st, recs, followed, bad = _follow(bm, None, Xd, m, n, k, s, T, seed, prec=prec,
                                           Xo=Xs, draws=cdraws)
    try:
        assert bad is None, "chunk %r: no admissible oracle outcome matches" % bad
        bm.bm_set_state(ctx, st.C.astype(np.float32), st.live.astype(np.uint8), st.f_opt, T)
        labels = torch.empty(m, dtype=torch.int32, device="cuda:0")
        sse = bm.bm_assign(ctx, labels)
    finally:
        bm.bm_destroy(ctx)
    lab_gpu = host(labels)
    base = "/dev/shm" if os.path.isdir("/dev/shm") else None
    with tempfile.TemporaryDirectory(dir=base) as tmp:
        path = os.path.join(tmp, "X.npy")
        np.save(path, Xd.cpu().numpy())
        del Xd
        torch.cuda.empty_cache()
        A, d1, d2 = pf.final_assignment_parallel(path, m, st.C, st.live)
    sse_ref = float(d1.sum())
    nbad, nties = labels_match(lab_gpu, A, d1, d2)
    assert nbad == 0 and rel(sse, sse_ref) <= OBJ_REL
    _report(name, chunks=T, followed=[list(f) for f in followed],
            accepted=sum(r.accepted for r in recs), lloyd_iters=sum(r.iters for r in recs),
            final_rows=m, final_tie_rows=nties, sse_rel=rel(sse, sse_ref))
    assert len(followed) <= max_followed


def test_c3_chunks_and_full_final_assignment(bm):
    m, n, k, s, seed = 10_000_000, 128, 50, 50_000, 0
    Xd = bi.mixtures.gas_sensor_like_device(seed, m=m, n=n, device="cuda:0")
    _follow_device_workload(bm, Xd, m, n, k, s, C3_CHUNKS, seed, 1,
                            "c3_gas_sensor_like_seed0", 4)


def test_c3_fp8_variant_chunks_and_full_final_assignment(bm):
    m, n, k, s, seed = 2_000_000, 384, 100, 50_000, 0
    Xd = bi.mixtures.scaled_384_device(seed, m=m, device="cuda:0")
    _follow_device_workload(bm, Xd, m, n, k, s, FP8_CHUNKS, seed, 2,
                            "c3_fp8_scaled_384_seed0", 6)
