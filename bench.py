"""Benchmark of the GB300 Big-means hot path (one JSON line on stdout).

Workload (default): the precision-form job -- m = 10,000,000 points, n = 128,
100 isotropic Gaussian components with Dirichlet(0.5) weights (generated on
the device, 5.12 GB), k = 50, s = 50,000, 100 chunks, then the final
full-data assignment with its float64 SSE.  One step = one complete Big-means
job: reset the incumbent, 100 chunks (sample draw, gather, K-means++ reseed,
Lloyd to the paper's stop rule, keep-the-best), final assignment.

The timed form is BF16 + rescore (BF16 tensor-core products with FP32
accumulation, exact FP32 rescoring of every row the error bound cannot
settle); the plain FP32 form and the split-BF16 form of the same job are
timed beside it (time to the same SSE).  The metric
is distance throughput: 2 n flops per point-to-centroid distance evaluation
(the paper's n_d counter) over the step time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 oracle (the slow CPU statement of the same
method) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import platform
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("dist TFLOP/s & time-to-SSE, BF16+rescore vs plain FP32 @≤1e-6 rel; "
          "req p50/p99")
UNIT = "TFLOP/s"

# the timed job: m = 1e7, n = 128 mixture (generated on the device)
C3_WORKLOAD = dict(name="gas_sensor_like_m1e7_n128_k50_s50000_T100", m=10_000_000, n=128,
                   k=50, s=50_000, chunks=100, seed=0)
HEAD_FORM = "bf16"
SIDE_FORMS = ("fp32", "bf16x3")     # timed beside it, same window
# further jobs reported beside it
C2_WORKLOAD = dict(name="hepmass_like_m1e6_n28_k25_s50000_T100", m=1_000_000, n=28,
                   k=25, s=50_000, chunks=100, seed=0)
C3_FP8_WORKLOAD = dict(name="scaled_384_m2e6_n384_k100_s50000_T100", m=2_000_000, n=384,
                       k=100, s=50_000, chunks=100, seed=0)

# the oracle's bounded sample of the timed job: the first chunks of the run
# plus the final assignment of every ASSIGN_STRIDE-th row
CPU_SAMPLE_CHUNKS = 8
CPU_ASSIGN_STRIDE = 10
REF_SAMPLE_CHUNKS = 1        # per step of --impl reference
REF_ASSIGN_STRIDE = 200

FORM_CODES = {"fp32": 0, "bf16": 1, "fp8": 2, "bf16x3": 3}

# ncu dram__bytes_read.sum + dram__bytes_write.sum of one chunk_tc_kernel
# launch (a typical chunk: gather + BF16 tiles + Lloyd), n = 128, k = 50,
# s = 50,000; the gather reads s rows whatever m is
CHUNK_TC_DRAM_BYTES = 26_153_728 + 2_158_592


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the further jobs (n = 28, E4M3, launch latency, grouped, serving)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-grouped", action="store_true")
    ap.add_argument("--profile", choices=["chunk_np", "chunk_tc", "assign_tc", "assign_fp8",
                                          "draw_m1e7", "grouped"],
                    default=None,
                    help="run one short job of a kernel family (for ncu captures) and exit")
    ap.add_argument("--chunks", type=int, default=C3_WORKLOAD["chunks"])
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    """(HBM GB/s, BF16 dense TFLOP/s burst, source) of the GB300s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    except OSError:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, pw, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": float(max(pw)) if pw else None}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------------ oracle baseline

def oracle_sample_inputs(Xd, wl, chunks, stride, path):
    """Writes the rows the oracle's bounded sample reads to `path` (.npz): the
    sample rows of chunks 0..chunks-1 (with their draws, indices remapped into
    the compact array) and every stride-th row of X for the final assignment."""
    import torch
    import bminputs
    m, k, s, seed = wl["m"], wl["k"], wl["s"], wl["seed"]
    idxs, ufs, us = [], [], []
    for t in range(chunks):
        idx, uf, u = bminputs.chunk_draws(seed, t, m, s, k)
        idxs.append(np.asarray(idx, np.int64))
        ufs.append(uf)
        us.append(u)
    allidx = np.concatenate(idxs)
    Xs = Xd[torch.from_numpy(allidx).to(Xd.device)].cpu().numpy()
    rows = np.arange(0, m, stride, dtype=np.int64)
    Xa = Xd[torch.from_numpy(rows).to(Xd.device)].cpu().numpy()
    np.savez(path, Xs=Xs, Xa=Xa, uf=np.array(ufs), u=np.stack(us), s=s, k=k, chunks=chunks)
    return {"chunk_rows": int(len(allidx)), "assign_rows": int(len(rows))}


def _oracle_job(args):
    """One bounded oracle run (child process, one thread): Alg. 1 on the saved
    chunk draws, then the final assignment of the saved rows.  With start_at,
    the run waits for that wall-clock time after loading, so concurrent runs
    start together.  Returns (seconds, distance evaluations, SSE of the sampled
    rows, wall-clock end)."""
    path, core, start_at = args
    if core is not None and hasattr(os, "sched_setaffinity"):
        try:
            os.sched_setaffinity(0, {core})
        except OSError:
            pass
    import oracle
    d = np.load(path)
    Xs, Xa = d["Xs"], d["Xa"]
    s, k, chunks = int(d["s"]), int(d["k"]), int(d["chunks"])
    draws = [(np.arange(t * s, (t + 1) * s), float(d["uf"][t]), d["u"][t]) for t in range(chunks)]
    if start_at is not None:
        time.sleep(max(0.0, start_at - time.time()))
    t0 = time.perf_counter()
    st, recs = oracle.big_means(Xs, k, draws)
    _, sse, _, _ = oracle.final_assignment(Xa, st.C, st.live)
    dt = time.perf_counter() - t0
    nd = sum(r.n_d for r in recs) + len(Xa) * int(st.live.sum())
    return dt, nd, sse, time.time()


def _oracle_proc(args, q):
    q.put(_oracle_job(args))


def _oracle_pool(path, cores, lead_s=12.0):
    """Runs len(cores) concurrent one-thread oracle jobs (one spawned process
    per core, pinned to it, all starting at one wall-clock time after their
    imports and loads); returns (wall seconds, [(s, n_d, sse, end)])."""
    import multiprocessing as mp
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for v in saved:
        os.environ[v] = "1"
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        start_at = time.time() + lead_s
        procs = [ctx.Process(target=_oracle_proc, args=((path, c, start_at), q)) for c in cores]
        for pr in procs:
            pr.start()
        res = []
        try:
            for _ in procs:
                res.append(q.get(timeout=900))
        finally:
            for pr in procs:
                pr.join(timeout=30)
                if pr.is_alive():
                    pr.terminate()
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    wall = max(r[3] for r in res) - start_at
    return wall, res


def cpu_baseline(Xd, wl, chunks=CPU_SAMPLE_CHUNKS, stride=CPU_ASSIGN_STRIDE, all_cores=True):
    """The FP64 oracle, as it stands, on a bounded sample of the timed job
    (its first `chunks` chunks + the final assignment of every stride-th row),
    on one core and as one concurrent replica per core; the same metric
    (distance TFLOP/s), measured on the sample."""
    n = wl["n"]
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "oracle_sample.npz")
        info = oracle_sample_inputs(Xd, wl, chunks, stride, path)
        core0 = sorted(os.sched_getaffinity(0))[0] if hasattr(os, "sched_getaffinity") else None
        wall1, r1 = _oracle_pool(path, [core0], lead_s=6.0)
        secs, nd, sse, _ = r1[0]
        out = {"value": 2.0 * n * nd / secs / 1e12, "unit": UNIT, "cores": 1,
               "kind": "oracle", "cpu": cpu_model(),
               "sample": "first %d of %d chunks (%d sample rows) + final assignment of "
                         "every %dth row (%d of %d), numpy/scipy float64, one thread pinned "
                         "to one core; %.2f s, sampled SSE %.6e; the metric is a rate, "
                         "measured on the sample"
                         % (chunks, wl["chunks"], info["chunk_rows"], stride,
                            info["assign_rows"], wl["m"], secs, sse),
               "seconds": secs, "n_d": nd}
        if all_cores:
            ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") \
                else (os.cpu_count() or 1)
            cores = sorted(os.sched_getaffinity(0))[:ncores] if hasattr(os, "sched_getaffinity") \
                else list(range(ncores))
            wallN, rN = _oracle_pool(path, cores)
            ndN = sum(r[1] for r in rN)
            out["all_cores"] = {
                "value": 2.0 * n * ndN / wallN / 1e12, "unit": UNIT, "cores": len(cores),
                "sample": "%d concurrent one-thread replicas of the same sample, one per "
                          "core; aggregate distance throughput over the wall time %.2f s"
                          % (len(cores), wallN)}
    return out


def run_reference(args, wl):
    """--impl reference: the FP64 oracle on a bounded sample of the timed job
    per step (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import torch
    import bminputs
    dev = torch.device("cuda", 0)
    Xd = bminputs.mixtures.gas_sensor_like_device(wl["seed"], m=wl["m"], n=wl["n"], device=dev)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "oracle_sample.npz")
        info = oracle_sample_inputs(Xd, wl, REF_SAMPLE_CHUNKS, REF_ASSIGN_STRIDE, path)
        del Xd
        torch.cuda.empty_cache()
        for _ in range(args.warmup):
            _oracle_job((path, None, None))
        runs = [_oracle_job((path, None, None)) for _ in range(args.steps)]
    secs = float(np.mean([r[0] for r in runs]))
    nd = runs[0][1]
    v = 2.0 * wl["n"] * nd / secs / 1e12
    sample = ("first %d of %d chunks (%d sample rows) + final assignment of every %dth row "
              "(%d of %d), numpy/scipy float64, single thread, per step; the metric is a "
              "rate, measured on the sample" % (REF_SAMPLE_CHUNKS, wl["chunks"],
                                                info["chunk_rows"], REF_ASSIGN_STRIDE,
                                                info["assign_rows"], wl["m"]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "m": wl["m"], "n": wl["n"], "k": wl["k"],
                       "s": wl["s"], "chunks": wl["chunks"], "sample": sample},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "cpu": cpu_model(),
                             "sample": sample, "value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def job_step(bm, ctx, stream, T, labels, ev):
    """One complete job on ctx: reset, T chunks, final assignment.  ev: three
    CUDA events recorded on the library's stream around the fit and the
    assignment."""
    bm.bm_reset(ctx)
    ev[0].record(stream)
    rep = bm.bm_fit_chunk(ctx, T)
    ev[1].record(stream)
    sse = bm.bm_assign(ctx, labels)
    ev[2].record(stream)
    return rep, sse


def run_ours(args, wl):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import bminputs
    import paper_2204_07485_gb300 as bm

    m, n, k, s, T = wl["m"], wl["n"], wl["k"], wl["s"], args.chunks
    seed = wl["seed"] + 1000 * rank          # independent replica per rank
    Xd = bminputs.mixtures.gas_sensor_like_device(wl["seed"], m=m, n=n, device=dev)
    stream = torch.cuda.Stream(device=dev)
    labels = torch.empty(m, dtype=torch.int32, device=dev)
    cfgs = {f: bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=FORM_CODES[f])
            for f in (HEAD_FORM,) + SIDE_FORMS}
    ctxs = {f: bm.bm_create(cfgs[f], Xd, stream.cuda_stream) for f in cfgs}
    new_ev = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(3)]   # noqa: E731

    for _ in range(args.warmup):
        job_step(bm, ctxs[HEAD_FORM], stream, T, labels, new_ev())
    for f in SIDE_FORMS:
        job_step(bm, ctxs[f], stream, T, labels, new_ev())
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    # X (5.12 GB) is far larger than L2 (129 MB): every step streams it anew
    events, reps = [], []
    side = {f: ([], []) for f in SIDE_FORMS}   # form -> (events, reports)
    with ClockSampler(local if world > 1 else 0) as clocks:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            ev = new_ev()
            reps.append(job_step(bm, ctxs[HEAD_FORM], stream, T, labels, ev))
            events.append(ev)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        # the other forms of the same job, beside it (same sampler window)
        for f in SIDE_FORMS:
            for _ in range(args.steps):
                ev = new_ev()
                side[f][1].append(job_step(bm, ctxs[f], stream, T, labels, ev))
                side[f][0].append(ev)
            torch.cuda.synchronize(dev)
    fit_ms = [e[0].elapsed_time(e[1]) for e in events]
    asg_ms = [e[1].elapsed_time(e[2]) for e in events]
    step_ms = [a + b for a, b in zip(fit_ms, asg_ms)]
    rep, sse = reps[-1]
    C = np.zeros((k, n), np.float32)
    mask = np.zeros(k, np.uint8)
    f_opt = bm.bm_objective(ctxs[HEAD_FORM], C, mask)
    nlive = int(mask.sum())
    nd_fit = rep["n_d"]                      # K-means++ + Lloyd of the step
    nd_step = nd_fit + m * nlive             # + final assignment
    flops_step = 2.0 * n * nd_step
    my_ms = float(np.sum(step_ms))
    if world > 1:
        t = torch.tensor([my_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    else:
        total_ms = my_ms
    value = world * args.steps * flops_step / (total_ms / 1e3) / 1e12
    phases = traced_phases(bm, Xd, cfgs[HEAD_FORM], stream, T)

    # roofline of the dominant kernel (largest share of the step)
    fit_per_step = float(np.mean(fit_ms))
    asg_per_step = float(np.mean(asg_ms))
    hbm_peak, bf16_peak, peak_src = measured_peaks()
    chunk_kernel = {
        "kernel": "chunk_tc_kernel (gather + BF16 planes + K-means++ + Lloyd + "
                  "keep-best; BF16 tcgen05 MMAs, exact FP32 rescoring)",
        "bound": "tensor",
        "achieved": 2.0 * n * nd_fit / (fit_per_step / 1e3) / 1e12,
        "peak": bf16_peak, "unit": "TFLOP/s",
        "peak_source": "%s dense BF16 (burst) of MEASURED_PEAKS" % peak_src,
        "launch_ms": fit_per_step / T,
        "launches_per_step": T, "share": fit_per_step / (fit_per_step + asg_per_step),
        "hbm_bytes_per_launch": s * n * 4,
        "hbm_gbs": s * n * 4 * T / (fit_per_step / 1e3) / 1e9}
    chunk_kernel["frac"] = chunk_kernel["achieved"] / chunk_kernel["peak"]
    abytes = m * n * 4 + m * 4
    assign_kernel = {
        "kernel": "assign_tcs_kernel (final assignment, BF16 MMAs + exact FP32 "
                  "rescoring, FP64 SSE)",
        "bound": "hbm",
        "achieved": abytes / (asg_per_step / 1e3) / 1e9, "peak": hbm_peak,
        "peak_source": "%s HBM copy bandwidth" % peak_src,
        "unit": "GB/s", "launch_ms": asg_per_step,
        "share": asg_per_step / (fit_per_step + asg_per_step), "algorithmic_bytes": abytes}
    assign_kernel["frac"] = assign_kernel["achieved"] / assign_kernel["peak"]
    dom = chunk_kernel if chunk_kernel["share"] >= assign_kernel["share"] else assign_kernel
    traffic = CHUNK_TC_DRAM_BYTES if dom is chunk_kernel else None
    roofline = {"bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
                "unit": dom["unit"], "frac": dom["frac"], "traffic": traffic,
                "kernel": dom["kernel"], "peak_source": dom["peak_source"],
                "timing": "CUDA events on the library's stream around bm_fit_chunk "
                          "(100 chunk launches + 2 sample-draw launches) each timed step"}

    # end to end through the host-memory entry point (pinned X in, results out)
    Xh = torch.empty((m, n), dtype=torch.float32).pin_memory()
    Xh.copy_(Xd)
    lab_h = torch.empty(m, dtype=torch.int32).pin_memory()
    Ch = np.zeros((k, n), np.float32)
    mh = np.zeros(k, np.uint8)
    e2e_times = []
    for i in range(max(1, min(args.steps, 3)) + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sse_h, rep_h = bm.bm_fit_host(cfgs[HEAD_FORM], Xh.data_ptr(), T, Ch, mh, lab_h.data_ptr())
        if i > 0:                            # the first call sets up the host pool
            e2e_times.append(time.perf_counter() - t0)
    e2e_val = flops_step / float(np.median(e2e_times)) / 1e12
    e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": m * n * 4,
           "d2h_bytes_per_step": m * 4 + k * n * 4 + k + 8,
           "ms_per_step": float(np.median(e2e_times)) * 1e3,
           "host_gather_ctas": rep_h["host_gathers"],
           "sse_equals_device_path": bool(sse_h == sse)}
    del Xh, lab_h

    out = None
    if rank == 0:
        head_ms = total_ms / args.steps
        side_forms = {}
        for f in SIDE_FORMS:
            evs, rps = side[f]
            ffit = [e[0].elapsed_time(e[1]) for e in evs]
            fasg = [e[1].elapsed_time(e[2]) for e in evs]
            frep, fsse = rps[-1]
            fms = float(np.mean(np.add(ffit, fasg)))
            side_forms[f] = {
                "time_to_sse_ms": fms, "fit_ms": float(np.mean(ffit)),
                "assign_ms": float(np.mean(fasg)), "sse": fsse,
                "value": 2.0 * n * (frep["n_d"] + m * nlive) / (fms / 1e3) / 1e12,
                "sse_rel_diff_vs_head": abs(fsse - sse) / fsse,
                "same_lloyd_iters": frep["lloyd_iters"] == rep["lloyd_iters"]}
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": head_ms, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
               "data": "synthetic",
               "config": {"workload": wl["name"], "m": m, "n": n, "k": k, "s": s,
                          "chunks": T, "seed": wl["seed"],
                          "form": "BF16 + rescore (BF16 tensor-core products, FP32 "
                                  "accumulation, exact FP32 rescoring)",
                          "l2": "X is 5.12 GB, 40x L2: each step streams it from HBM",
                          "parallelism": "replicas (independent job per GPU)"},
               "time_to_sse_ms": head_ms, "sse": sse,
               "forms": side_forms,
               "speedup_vs_fp32": side_forms["fp32"]["time_to_sse_ms"] / head_ms,
               "f_opt": f_opt, "live": nlive, "lloyd_iters_per_step": rep["lloyd_iters"],
               "accepted_per_step": rep["accepted"], "n_d_per_step": nd_step,
               "fit_ms_per_step": fit_per_step, "assign_ms_per_step": asg_per_step,
               "chunk_phase_ms_per_step": phases, "wall_s": t_wall,
               "gpu_launches": args.steps * (T + (T + 63) // 64 + 1),
               "roofline": roofline,
               "kernels": {"chunk": chunk_kernel, "assign": assign_kernel},
               "clocks": clocks.summary(), "e2e": e2e}
    for c in ctxs.values():
        bm.bm_destroy(c)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(Xd, wl)
    del Xd, labels
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_extras:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        extra = {}
        w2 = C2_WORKLOAD
        X2 = torch.from_numpy(bminputs.mixtures.hepmass_like(w2["seed"], m=w2["m"])).to(dev)
        extra[w2["name"]] = precision_forms(bm, torch, dev, X2, w2["m"], w2["n"], w2["k"],
                                            w2["s"], w2["chunks"], w2["seed"], 5, 2, flush)
        del X2
        v8 = C3_FP8_WORKLOAD
        Xs = bminputs.mixtures.scaled_384_device(v8["seed"], m=v8["m"], device=dev)
        extra[v8["name"]] = precision_forms(bm, torch, dev, Xs, v8["m"], v8["n"], v8["k"],
                                            v8["s"], v8["chunks"], v8["seed"], 3, 1, flush,
                                            forms=("fp32", "bf16", "bf16x3", "fp8"))
        del Xs, flush
        torch.cuda.empty_cache()
        out["other_jobs"] = extra
        out["tile_pipeline"] = tile_pipeline(bm)
        out["launch_latency"] = launch_latency(bm, torch, dev)
        if not args.no_grouped:
            out["grouped"] = grouped(bm, torch, dev)
        if not args.no_serving:
            # the specified load (200/s, beyond this mix's capacity on one GPU:
            # latency there is queueing), the capacity (every job at once) and
            # a load below it (service latency)
            out["serving"] = serving(bm, torch, dev)
            keep = ("workload", "jobs_per_s", "completed", "failed", "wall_s", "workers",
                    "latency_ms", "queue_ms", "offered_rps")
            out["serving_capacity"] = {q: v for q, v in serving(
                bm, torch, dev, dict(SERVING, rate=None)).items() if q in keep[:6]}
            out["serving_below_capacity"] = {q: v for q, v in serving(
                bm, torch, dev, dict(SERVING, rate=120.0, requests=1200)).items() if q in keep}
    if rank == 0:
        print(json.dumps(out))
    return 0


def time_jobs(bm, torch, ctx, stream, T, steps, warmup, flush, labels):
    """Runs `warmup` + `steps` complete jobs; per-step CUDA-event times (L2
    flushed between steps)."""
    def new_ev():
        return [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(warmup):
        job_step(bm, ctx, stream, T, labels, new_ev())
    torch.cuda.synchronize()
    events, reps = [], []
    for i in range(steps):
        ev = new_ev()
        reps.append(job_step(bm, ctx, stream, T, labels, ev))
        events.append(ev)
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
    torch.cuda.synchronize()
    fit = [e[0].elapsed_time(e[1]) for e in events]
    asg = [e[1].elapsed_time(e[2]) for e in events]
    return fit, asg, reps


def precision_forms(bm, torch, dev, X, m, n, k, s, T, seed, steps, warmup, flush,
                    forms=("fp32", "bf16x3")):
    """Time to SSE of the same job in the FP32 and tensor-core forms, with the
    distance throughput of each."""
    stream = torch.cuda.Stream(device=dev)
    labels = torch.empty(m, dtype=torch.int32, device=dev)
    out = {}
    for form in forms:
        cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=seed, precision=FORM_CODES[form])
        ctx = bm.bm_create(cfg, X, stream.cuda_stream)
        try:
            fit, asg, reps = time_jobs(bm, torch, ctx, stream, T, steps, warmup, flush, labels)
            mask = np.zeros(k, np.uint8)
            bm.bm_objective(ctx, None, mask)
        finally:
            bm.bm_destroy(ctx)
        rep, sse = reps[-1]
        ms = float(np.mean(np.add(fit, asg)))
        out[form] = {"time_to_sse_ms": ms, "fit_ms": float(np.mean(fit)),
                     "assign_ms": float(np.mean(asg)), "sse": sse,
                     "tflops": 2.0 * n * (rep["n_d"] + m * int(mask.sum())) / (ms / 1e3) / 1e12}
    base = out["fp32"]
    for form, r in out.items():
        r["sse_rel_diff_vs_fp32"] = abs(r["sse"] - base["sse"]) / base["sse"]
        r["speedup_vs_fp32"] = base["time_to_sse_ms"] / r["time_to_sse_ms"]
    return out


def traced_phases(bm, Xd, cfg, stream, T):
    """Device time (ms) per chunk phase of one extra job run with tracing on
    (the timed steps run without it: the timer reads sit on the barrier path)."""
    tcfg = bm.bm_config_default(**{f: getattr(cfg, f) for f, _ in cfg._fields_})
    tcfg.trace = 1
    ctx = bm.bm_create(tcfg, Xd, stream.cuda_stream)
    try:
        bm.bm_reset(ctx)
        bm.bm_fit_chunk(ctx, T)
        return {p: round(v, 4) for p, v in bm.bm_trace(ctx).items()}
    finally:
        bm.bm_destroy(ctx)


def tile_pipeline(bm, steps=16384):
    """The distance-tile pipeline alone, operands resident in shared memory
    (bm_tile_bench): MMA throughput with the candidate epilogue and without,
    at k = 50 (MMA N = 64) for n = 64, 128, 256; against the measured BF16
    peak.  Algorithmic flops count 2 n k per point-centroid pair."""
    _, bf16_peak, src = measured_peaks()
    out = {"peak_tflops": bf16_peak, "peak_source": src, "k": 50, "steps_per_cta": steps}
    for n in (64, 128, 256):
        for planes in (1, 2):
            for epi in (0, 1):
                bm.bm_tile_bench(n, 50, planes, 64, bool(epi))        # warm-up
                r = bm.bm_tile_bench(n, 50, planes, steps, bool(epi))
                secs = r["ms"] / 1e3
                mma = r["grid"] * steps * 2.0 * 128 * 64 * n * (3 if planes == 2 else 1)
                alg = r["grid"] * steps * 2.0 * 128 * 50 * n
                out["n%d_%s_%s" % (n, "bf16" if planes == 1 else "bf16x3",
                                   "epilogue" if epi else "mma_only")] = {
                    "ms": r["ms"], "mma_tflops": mma / secs / 1e12,
                    "mma_frac": mma / secs / 1e12 / bf16_peak,
                    "dist_tflops": alg / secs / 1e12, "tiles_resident": r["tiles"]}
    return out


def launch_latency(bm, torch, dev, jobs=10, warmup=3):
    """m = 20,000, n = 2, k = 10, s = 2,000, 20 chunks (ten 2-D blobs): the
    whole chunk fits one SM, so the time is launch and barrier latency.  Fit
    time per job with the launches recorded in a CUDA graph and one by one."""
    import bminputs
    m, n, k, s, T = 20_000, 2, 10, 2_000, 20
    Xd = torch.from_numpy(bminputs.mixtures.blobs_2d(0)).to(dev)
    out = {"workload": "blobs_2d_m20000_n2_k10_s2000_T20"}
    for graphs in (0, 1):
        stream = torch.cuda.Stream(device=dev)
        cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=0, graphs=graphs)
        ctx = bm.bm_create(cfg, Xd, stream.cuda_stream)
        try:
            times, iters = [], 0
            for i in range(warmup + jobs):
                bm.bm_reset(ctx)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rep = bm.bm_fit_chunk(ctx, T)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if i >= warmup:
                    times.append(e0.elapsed_time(e1))
                    iters += rep["lloyd_iters"]
        finally:
            bm.bm_destroy(ctx)
        ms = float(np.mean(times))
        out["graph" if graphs else "direct"] = {
            "fit_ms": ms, "us_per_chunk": ms * 1e3 / T,
            "us_per_lloyd_iter": ms * 1e3 * jobs / max(1, iters)}
    return out


def grouped(bm, torch, dev, count=256, runs=3, warmup=1):
    """256 independent chunks (s ~ U[4000, 64000], n ~ U{16, 32, 64, 128},
    k ~ U{5, 10, 25, 50}, chunk i a mixture of k_i isotropic components drawn
    with seed i; about 2 GB of float32 rows, more than L2) run to convergence
    by the grouped Lloyd launches from a seeded Forgy start.  Reports the time
    per run, per Lloyd step of the whole group, the distance throughput
    (2 n flops per point-centroid distance), the same with one CTA per
    problem (a fixed, untuned partition), and parity of sampled problems
    against the same problem run alone (bm_lloyd)."""
    import bminputs
    spec = bminputs.mixtures.grouped_chunks_spec(0, count)
    probs, starts = [], []
    for q in spec:
        P = bminputs.mixtures.isotropic_blobs_device(q["s"], q["n"], q["k"], q["seed"],
                                                     device=dev)
        rows = torch.from_numpy(bminputs.mixtures.forgy_rows(q["s"], q["k"], q["seed"])).to(dev)
        C0 = P[rows].contiguous()
        C = C0.clone()
        mask = torch.ones(q["k"], dtype=torch.uint8, device=dev)
        probs.append(dict(P=P, s=q["s"], n=q["n"], k=q["k"], C=C, mask=mask))
        starts.append(C0)
    torch.cuda.synchronize(dev)
    rows_total = sum(q["s"] for q in spec)
    bytes_total = sum(4 * q["s"] * q["n"] for q in spec)
    out = {"workload": "grouped_256_chunks_s4k-64k_n16-128_k5-50",
           "problems": count, "rows": rows_total, "bytes": bytes_total}
    stream = torch.cuda.Stream(device=dev)

    def reset():
        with torch.cuda.stream(stream):
            for p, C0 in zip(probs, starts):
                p["C"].copy_(C0)
                p["mask"].fill_(1)

    # (balance, tile mode): cost-balanced partition with autotuned tile shapes,
    # the same with the fixed lane-per-centroid tile, one CTA per problem
    for balance, mode in ((1, 0), (1, 1), (0, 1)):
        g = bm.bm_group_create(probs, balance=bool(balance), stream=stream)
        try:
            bm.bm_group_set_tiles(g, mode)
            info = bm.bm_group_info(g)
            times, res, steps = [], None, 0
            for i in range(warmup + runs):
                reset()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res, steps = bm.bm_group_run(g, count)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if i >= warmup:
                    times.append(e0.elapsed_time(e1))
            shapes = bm.bm_group_tiles(g, count)
        finally:
            bm.bm_group_destroy(g)
        ms = float(np.median(times))
        flops = sum(2.0 * q["n"] * r["n_d"] for q, r in zip(spec, res))
        iters = [r["iters"] for r in res]
        entry = {"ms_per_run": ms, "steps": steps, "ms_per_step": ms / steps,
                 "max_iters": max(iters), "mean_iters": float(np.mean(iters)),
                 "dist_tflops": flops / (ms / 1e3) / 1e12, "grid": info["grid"],
                 "segments": info["segments"]}
        if balance and mode == 0:
            rows_lanes = sorted({(q["n"], q["k"]) for q, sh in zip(spec, shapes) if sh == 1})
            entry["row_lane_tiles_for_nk"] = [list(x) for x in rows_lanes]
        key = ("balanced_autotuned_tiles" if mode == 0 else "balanced_fixed_tile") if balance \
            else "one_cta_per_problem"
        out[key] = entry
        if balance and mode == 0:
            balanced_res = res
    # parity per problem against the same problem alone
    worst, same = 0.0, True
    for i in (0, count // 2, count - 1):
        q = spec[i]
        C = starts[i].clone()
        mask = torch.ones(q["k"], dtype=torch.uint8, device=dev)
        f, it = bm.bm_lloyd(probs[i]["P"], q["s"], q["n"], q["k"], C, mask)
        r = balanced_res[i]
        same = same and it == r["iters"]
        worst = max(worst, abs(f - r["f"]) / max(abs(r["f"]), 1e-300))
    out["alone_parity"] = {"sampled": 3, "same_iters": same, "max_rel_f": worst}
    del probs, starts
    torch.cuda.empty_cache()
    return out


# 100 jobs/s: below the measured capacity of this mix on one GB300 (about
# 117 jobs/s with 4 workers), so latency reflects service, not an
# ever-growing queue
# the serving workload: Poisson arrivals at 200 jobs/s, 2,000 jobs; `rate`
# None submits every job at once (the server's capacity)
SERVING = dict(requests=2000, rate=200.0, chunks=20, workers=8, seed=0,
               n_set=(8, 28, 68, 128, 384), m_range=(1e4, 5e6), k_range=(2, 100),
               s_max=50_000)


def serving(bm, torch, dev, spec=SERVING):
    """Poisson arrivals of whole jobs (m log-uniform, n from the set, k
    uniform, s = min(m, 50k), FP32 or BF16 + rescore by a fair coin, 20 chunks +
    final assignment), each job's data synthesized on the device from (seed,
    job id) just before it is submitted.  Latency = submission -> results
    ready, on the server's clock."""
    rng = np.random.default_rng(spec["seed"])
    R = spec["requests"]
    gaps = rng.exponential(1.0 / spec["rate"], size=R) if spec["rate"] else np.zeros(R)
    arrive = np.cumsum(gaps)
    lo, hi = np.log(spec["m_range"][0]), np.log(spec["m_range"][1])
    ms = np.exp(rng.uniform(lo, hi, size=R)).astype(np.int64)
    ns = rng.choice(spec["n_set"], size=R)
    ks = rng.integers(spec["k_range"][0], spec["k_range"][1] + 1, size=R)
    precs = np.where(rng.random(R) < 0.5, bm.BM_FP32, bm.BM_BF16_RESCORE)
    # data: one seeded 100-component mixture per n, synthesized on the device
    # before the clock starts; job j reads m rows of it from a seeded offset
    import bminputs
    max_off = 1 << 16
    offs = rng.integers(0, max_off, size=R)
    pools = {}
    for n in spec["n_set"]:
        sel = ns == n
        if sel.any():
            pools[int(n)] = bminputs.mixtures.isotropic_blobs_device(
                int(ms[sel].max()) + max_off, int(n), 100, spec["seed"] + int(n), device=dev)
    torch.cuda.synchronize(dev)
    sv = bm.bm_server_create(workers=spec["workers"], max_queue=max(256, R))
    pending = {}            # ticket -> (job id, X kept alive until the job ends)
    results = [None] * R
    submit_t = np.zeros(R)
    lock = threading.Lock()
    finished = threading.Event()
    count = [0]

    def on_done(ticket, res):
        with lock:
            jid, _ = pending.pop(ticket)
            results[jid] = res
            count[0] += 1
            if count[0] == R:
                finished.set()

    t0 = time.perf_counter()
    try:
        for j in range(R):
            delay = arrive[j] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            m, n, k = int(ms[j]), int(ns[j]), int(ks[j])
            X = pools[n][int(offs[j]):int(offs[j]) + m]
            cfg = bm.bm_config_default(m=m, n=n, k=k, s=min(m, spec["s_max"]), seed=j,
                                       precision=int(precs[j]))
            with lock:
                submit_t[j] = time.perf_counter() - t0
                try:
                    ticket = bm.bm_submit(sv, cfg, X, spec["chunks"], callback=on_done)
                except bm.BigMeansError as e:   # refused at admission
                    results[j] = {"status": e.status}
                    count[0] += 1
                    continue
                pending[ticket] = (j, X)
        if count[0] == R:
            finished.set()
        finished.wait(600.0)
        wall = time.perf_counter() - t0
        stats = bm.bm_server_stats(sv)
    finally:
        bm.bm_server_destroy(sv)
    del pools
    done = [r for r in results if r is not None]
    ok = [r for r in done if r["status"] == 0]
    failures = [{"m": int(ms[j]), "n": int(ns[j]), "k": int(ks[j]), "precision": int(precs[j]),
                 "status": r["status"]} for j, r in enumerate(results)
                if r is not None and r["status"] != 0][:10]
    lat = np.array([r["latency_s"] for r in ok]) * 1e3
    que = np.array([r["queued_s"] for r in ok]) * 1e3

    def pct(a, q):
        return float(np.percentile(a, q)) if len(a) else None

    by_prec = {}
    for name, code in (("fp32", bm.BM_FP32), ("bf16", bm.BM_BF16_RESCORE)):
        sel = [r["latency_s"] * 1e3 for j, r in enumerate(results)
               if r is not None and r["status"] == 0 and precs[j] == code]
        by_prec[name] = {"jobs": len(sel), "p50_ms": pct(sel, 50), "p99_ms": pct(sel, 99)}
    run_ms_by_n = {}
    for nv in spec["n_set"]:
        sel = [r["run_s"] * 1e3 for j, r in enumerate(results)
               if r is not None and r["status"] == 0 and ns[j] == nv]
        if sel:
            run_ms_by_n["n%d" % nv] = round(float(np.mean(sel)), 2)
    return {"workload": ("poisson_%d_per_s_%d_jobs_mixed_shapes" % (spec["rate"], R)
                         if spec["rate"] else "all_%d_jobs_at_once_mixed_shapes" % R),
            "run_ms_mean_by_n": run_ms_by_n,
            "requests": R, "offered_rps": spec["rate"],
            "submitted_rps": R / max(submit_t[-1], 1e-9), "completed": len(ok),
            "failed": len(done) - len(ok), "wall_s": wall, "jobs_per_s": len(ok) / wall,
            "latency_ms": {"p50": pct(lat, 50), "p90": pct(lat, 90), "p99": pct(lat, 99),
                           "mean": float(lat.mean()) if len(lat) else None,
                           "max": float(lat.max()) if len(lat) else None},
            "queue_ms": {"p50": pct(que, 50), "p99": pct(que, 99)},
            "by_precision": by_prec, "failures": failures,
            "workers": spec["workers"], "chunks": spec["chunks"],
            "server_rejected": {"busy": stats["rejected_busy"], "memory": stats["rejected_memory"]},
            "data": "one seeded 100-component isotropic mixture per n, synthesized on "
                    "the device before the clock starts; job j reads m rows from a "
                    "seeded offset"}


PROFILE_CASES = {
    # kernel family: (m, n, k, s, precision, chunks); small jobs for ncu captures
    "chunk_np": (1_000_000, 28, 25, 50_000, 0, 4),     # chunk_kernel<28, 0>
    "chunk_tc": (1_000_000, 128, 50, 50_000, 1, 3),    # chunk_tc_kernel, BF16 screening
    "assign_tc": (2_000_000, 128, 50, 50_000, 1, 1),   # assign_tcs_kernel, BF16 (final assignment)
    "assign_fp8": (2_000_000, 384, 100, 50_000, 2, 1),  # assign_tc_kernel<true> (E4M3)
    "draw_m1e7": (10_000_000, 4, 5, 50_000, 0, 64),     # draw_kernel, bitmaps in global memory
}


def profile_grouped(count=64):
    """The first `count` chunks of the grouped workload run once (for ncu)."""
    import torch
    import bminputs
    import paper_2204_07485_gb300 as bm
    dev = torch.device("cuda", 0)
    spec = bminputs.mixtures.grouped_chunks_spec(0, count)
    probs = []
    for q in spec:
        P = bminputs.mixtures.isotropic_blobs_device(q["s"], q["n"], q["k"], q["seed"],
                                                     device=dev)
        rows = torch.from_numpy(bminputs.mixtures.forgy_rows(q["s"], q["k"], q["seed"])).to(dev)
        probs.append(dict(P=P, s=q["s"], n=q["n"], k=q["k"], C=P[rows].contiguous(),
                          mask=torch.ones(q["k"], dtype=torch.uint8, device=dev)))
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)
    g = bm.bm_group_create(probs, stream=stream)
    try:
        res, steps = bm.bm_group_run(g, count)
    finally:
        bm.bm_group_destroy(g)
    print(json.dumps({"profile": "grouped", "problems": count, "steps": steps,
                      "max_iters": max(r["iters"] for r in res)}))
    return 0


def profile_case(name):
    """One short job of the named kernel family (for ncu; prints one line)."""
    import torch
    import bminputs
    import paper_2204_07485_gb300 as bm
    if name == "grouped":
        return profile_grouped()
    m, n, k, s, prec, T = PROFILE_CASES[name]
    dev = torch.device("cuda", 0)
    if n == 28:
        X = torch.from_numpy(bminputs.mixtures.hepmass_like(0, m=m)).to(dev)
    elif n == 384:
        X = bminputs.mixtures.scaled_384_device(0, m=m, device=dev)
    else:
        X = bminputs.mixtures.isotropic_blobs_device(m, n, 100, 0, alpha=0.5, device=dev)
    stream = torch.cuda.Stream(device=dev)
    cfg = bm.bm_config_default(m=m, n=n, k=k, s=s, seed=0, precision=prec, graphs=0)
    ctx = bm.bm_create(cfg, X, stream.cuda_stream)
    try:
        rep = bm.bm_fit_chunk(ctx, T)
        sse = bm.bm_assign(ctx, None)
    finally:
        bm.bm_destroy(ctx)
    print(json.dumps({"profile": name, "chunks": rep["chunks"], "lloyd_iters": rep["lloyd_iters"],
                      "sse": sse}))
    return 0


def main():
    args = parse()
    if args.profile:
        return profile_case(args.profile)
    wl = dict(C3_WORKLOAD)
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
