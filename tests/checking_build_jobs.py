"""Jobs run by a child process against one build of the library (the product
build, or one of the checking builds selected through BM_LIBRARY: device
index guards, or host AddressSanitizer + UndefinedBehaviorSanitizer).

  python tests/checking_build_jobs.py host   # entry points that need no GPU
  python tests/checking_build_jobs.py gpu    # one small job of every kernel family

Prints one JSON object of results; the tests compare the objects of the
builds with each other.  Inputs are seeded.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402


def host_jobs(bm):
    out = {}
    cfg = bm.bm_config_default(m=1000, n=4, k=3, s=100)
    out["defaults"] = [cfg.max_iter, cfg.tol, cfg.kpp_trials, cfg.graphs]
    out["status"] = [bm.bm_status_string(i) for i in range(10)]
    bad = bm.bm_config_default(m=10, n=4, k=20, s=5)   # k > s
    try:
        bm.bm_create(bad, 1 << 20)
        out["create_bad"] = "accepted"
    except bm.BigMeansError as e:
        out["create_bad"] = e.status
    out["late_reads"] = bm.bm_sync_late_reads()
    return out


def gpu_jobs(bm):
    import torch
    import bminputs as bi
    dev = torch.device("cuda", 0)
    out = {}

    def job(name, X, m, n, k, s, T, prec=0, **kw):
        Xd = torch.from_numpy(X).to(dev)
        cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=3, precision=prec, **kw)
        ctx = bm.bm_create(cfg, Xd)
        try:
            rep = bm.bm_fit_chunk(ctx, T)
            labels = torch.empty(m, dtype=torch.int32, device=dev)
            sse = bm.bm_assign(ctx, labels)
            C = np.zeros((k, n), np.float32)
            mask = np.zeros(k, np.uint8)
            f = bm.bm_objective(ctx, C, mask)
        finally:
            bm.bm_destroy(ctx)
        out[name] = {"sse": sse, "f_opt": f, "n_d": rep["n_d"], "iters": rep["lloyd_iters"],
                     "labels": int(labels.to(torch.int64).sum().item()),
                     "C": float(np.float64(C).sum())}

    X2, _ = bi.mixtures.isotropic_blobs(20_000, 2, 10, 0)
    job("np_n2", X2, 20_000, 2, 10, 2_000, 5)
    X28 = bi.mixtures.hepmass_like(1, m=200_000)
    job("np_n28", X28, 200_000, 28, 25, 20_000, 3)
    X64, _ = bi.mixtures.isotropic_blobs(20_000, 64, 40, 1)
    job("tiled_n64", X64, 20_000, 64, 33, 6_000, 3)
    X128, _ = bi.mixtures.isotropic_blobs(30_000, 128, 60, 2)
    job("tc_bf16", X128, 30_000, 128, 50, 6_000, 3, prec=1)
    job("tc_bf16x3", X128, 30_000, 128, 50, 6_000, 3, prec=3)
    X384, _ = bi.mixtures.isotropic_blobs(6_000, 384, 100, 3)
    job("tc_fp8", X384, 6_000, 384, 100, 3_000, 2, prec=2)
    job("forgy_keep", X64, 20_000, 64, 20, 4_000, 3, init=1, empty=1)

    # sample plan with the bitmap in global memory (m > 1.6 million)
    idx = torch.empty(5_000, dtype=torch.int32, device=dev)
    sums = []
    for t in range(3):
        bm.bm_draw_chunk(2_000_003, 5_000, 7, t, idx)
        sums.append(int(idx.to(torch.int64).sum().item()))
    out["draw_global"] = sums

    # step-level entry points
    P = torch.from_numpy(X128[:4_000]).to(dev)
    C0 = torch.zeros((50, 128), dtype=torch.float32, device=dev)
    m0 = torch.zeros(50, dtype=torch.uint8, device=dev)
    bm.bm_kpp_reseed(P, 4_000, 128, 50, C0, m0, 5, 0, 3)
    f, it = bm.bm_lloyd(P, 4_000, 128, 50, C0, m0)
    out["ops"] = {"lloyd_f": f, "iters": it, "C": float(C0.double().sum().item())}
    # every slot degenerate on the tiled FP32 kernel (12 CTAs): CTA 0 fills
    # slot 0 before the launch's first grid barrier while the others read
    # the starting centroids; the checking build's start skew exposes any
    # overlap of the two
    Xs, _ = bi.mixtures.isotropic_blobs(6_000, 128, 50, 2)
    idx_s, _, _ = bi.chunk_draws(2, 0, 6_000, 3_000, 50)
    Ps = torch.from_numpy(Xs[idx_s]).to(dev)
    Cs = torch.zeros((50, 128), dtype=torch.float32, device=dev)
    ms = torch.zeros(50, dtype=torch.uint8, device=dev)
    bm.bm_kpp_reseed(Ps, 3_000, 128, 50, Cs, ms, 2, 0, 3)
    out["kpp_all_degenerate"] = [float(v) for v in Cs.double().sum(dim=1).cpu().numpy()]
    out["assign_rows"] = bm.bm_assign_rows(P, 4_000, 128, C0, m0, 50)
    X28d = torch.from_numpy(X28[:50_000]).to(dev)
    C28 = torch.from_numpy(X28[:25].copy()).to(dev)
    m28 = torch.ones(25, dtype=torch.uint8, device=dev)
    out["noalloc"] = bm.bm_assign_rows_noalloc(X28d, 50_000, 28, C28, m28, 25)

    # host-memory entry point, workers, polish, streaming
    Xh = torch.from_numpy(X28).pin_memory()
    cfg = bm.bm_config_default(m=200_000, n=28, k=25, s=20_000, seed=4)
    sse_h, rep_h = bm.bm_fit_host(cfg, Xh.data_ptr(), 3)
    out["fit_host"] = {"sse": sse_h, "n_d": rep_h["n_d"]}
    Xd = torch.from_numpy(X28).to(dev)
    ctx = bm.bm_create(cfg, Xd)
    try:
        bm.bm_fit_workers(ctx, 2, 2, 1)
        pf, pit = bm.bm_polish(ctx, 5, 1e-4)
        out["workers_polish"] = {"f": pf, "iters": pit}
    finally:
        bm.bm_destroy(ctx)
    sctx = bm.bm_stream_create(cfg)
    try:
        for q in range(2):
            bm.bm_stream_push(sctx, Xd[q * 20_000:(q + 1) * 20_000], 20_000)
        out["stream"] = bm.bm_objective(sctx)
    finally:
        bm.bm_destroy(sctx)

    # grouped problems
    probs = []
    for i, (s, n, k) in enumerate([(3_000, 16, 5), (5_000, 64, 25), (2_000, 128, 10)]):
        Pi, _ = bi.mixtures.isotropic_blobs(s, n, k, 10 + i)
        Pd = torch.from_numpy(Pi).to(dev)
        probs.append(dict(P=Pd, s=s, n=n, k=k, C=Pd[:k].clone(),
                          mask=torch.ones(k, dtype=torch.uint8, device=dev)))
    g = bm.bm_group_create(probs)
    try:
        res, steps = bm.bm_group_run(g, len(probs))
    finally:
        bm.bm_group_destroy(g)
    out["grouped"] = [r["f"] for r in res]

    # the job server
    sv = bm.bm_server_create(workers=2)
    try:
        tickets = []
        for j in range(4):
            c = bm.bm_config_default(m=50_000, n=28, k=10 + j, s=10_000, seed=j)
            tickets.append(bm.bm_submit(sv, c, Xd[:50_000], 3))
        out["server"] = [bm.bm_wait(sv, t, 60.0)["sse"] for t in tickets]
    finally:
        bm.bm_server_destroy(sv)
    out["late_reads"] = bm.bm_sync_late_reads()
    return out


def main():
    import paper_2204_07485_gb300 as bm
    mode = sys.argv[1] if len(sys.argv) > 1 else "host"
    res = host_jobs(bm) if mode == "host" else gpu_jobs(bm)
    print(json.dumps(res, sort_keys=True))


if __name__ == "__main__":
    main()
