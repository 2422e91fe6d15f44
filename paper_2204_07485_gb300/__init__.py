"""Python binding of libbigmeans.so (GB300 Big-means, arXiv 2204.07485).

Argument marshalling only: every step of the clustering runs in the CUDA
library through its C ABI (``include/bigmeans.h``); the functions here carry
the same names.  Pointer arguments accept a plain integer address or any
object with ``data_ptr()`` (e.g. a torch tensor); streams accept an integer
handle or an object with ``cuda_stream``.  There is no CPU fallback: if the
shared library has not been built, importing this package raises.
"""
import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# BM_LIBRARY names a checking build of the same sources (the tests' index-
# guard and sanitizer variants); by default the in-tree product library.
LIB_PATH = os.environ.get("BM_LIBRARY") or os.path.join(_HERE, "libbigmeans.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libbigmeans.so is not built (expected at %s); run "
        "`python -c 'import __graft_entry__ as g; g.build()'` first" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

BM_OK, BM_EINVAL, BM_ENOMEM, BM_ECUDA, BM_ETIMEOUT, BM_EBUSY, BM_ECANCELLED, \
    BM_EUNSUPPORTED, BM_EGUARD = range(9)
BM_FP32, BM_BF16_RESCORE, BM_FP8_RESCORE, BM_BF16X3_RESCORE = range(4)
BM_INIT_KMEANSPP, BM_INIT_FORGY = 0, 1
BM_EMPTY_DEGENERATE, BM_EMPTY_KEEP = 0, 1


class bm_config(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int32), ("k", ctypes.c_int32),
                ("s", ctypes.c_int64), ("max_iter", ctypes.c_int32),
                ("tol", ctypes.c_double), ("kpp_trials", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("time_budget_s", ctypes.c_double), ("graphs", ctypes.c_int32),
                ("trace", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("init", ctypes.c_int32), ("empty", ctypes.c_int32)]


class bm_fit_report(ctypes.Structure):
    _fields_ = [("chunks", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("lloyd_iters", ctypes.c_int64), ("n_d", ctypes.c_int64),
                ("chunk_counter", ctypes.c_int64), ("f_opt", ctypes.c_double),
                ("seconds", ctypes.c_double), ("host_gathers", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class bm_server_config(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("max_queue", ctypes.c_int32), ("job_ctas", ctypes.c_int32)]


class bm_job_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sse", ctypes.c_double),
                ("f_opt", ctypes.c_double), ("lloyd_iters", ctypes.c_int64),
                ("accepted", ctypes.c_int64), ("queued_s", ctypes.c_double),
                ("run_s", ctypes.c_double), ("latency_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


bm_job_callback = ctypes.CFUNCTYPE(None, ctypes.c_uint64, ctypes.POINTER(bm_job_result),
                                   ctypes.c_void_p)


class bm_job(ctypes.Structure):
    _fields_ = [("cfg", bm_config), ("X_dev", ctypes.c_void_p), ("chunks", ctypes.c_int32),
                ("labels_dev", ctypes.c_void_p), ("C_out_host", ctypes.c_void_p),
                ("mask_out_host", ctypes.c_void_p), ("callback", bm_job_callback),
                ("user", ctypes.c_void_p)]


class bm_server_stats_t(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("submitted", "completed", "failed", "cancelled", "rejected_busy",
                 "rejected_memory", "queued", "running", "memory_in_use", "memory_budget")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class bm_group_problem(ctypes.Structure):
    _fields_ = [("P_dev", ctypes.c_void_p), ("s", ctypes.c_int64), ("n", ctypes.c_int32),
                ("k", ctypes.c_int32), ("C_dev", ctypes.c_void_p), ("mask_dev", ctypes.c_void_p),
                ("labels_dev", ctypes.c_void_p)]


class bm_group_result(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("n_d", ctypes.c_int64), ("iters", ctypes.c_int32),
                ("live", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BigMeansError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, bm_status_string(status), status))


_vp, _i32, _i64, _u64, _dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_uint64, ctypes.c_double)
_P = ctypes.POINTER

_SIGS = {
    "bm_config_default": (None, [_P(bm_config)]),
    "bm_status_string": (ctypes.c_char_p, [_i32]),
    "bm_create": (_i32, [_P(bm_config), _vp, _vp, _P(_vp)]),
    "bm_destroy": (_i32, [_vp]),
    "bm_reset": (_i32, [_vp]),
    "bm_fit_chunk": (_i32, [_vp, _i32, _P(bm_fit_report)]),
    "bm_assign": (_i32, [_vp, _vp, _P(_dbl)]),
    "bm_objective": (_i32, [_vp, _P(_dbl), _vp, _vp]),
    "bm_get_state": (_i32, [_vp, _vp, _vp, _P(_dbl), _P(_i64)]),
    "bm_set_state": (_i32, [_vp, _vp, _vp, _dbl, _i64]),
    "bm_trace": (_i32, [_vp, _P(_dbl), _i32]),
    "bm_polish": (_i32, [_vp, _i32, _dbl, _P(_dbl), _P(_i32)]),
    "bm_fit_workers": (_i32, [_vp, _i32, _i32, _i32, _P(bm_fit_report)]),
    "bm_stream_create": (_i32, [_P(bm_config), _vp, _P(_vp)]),
    "bm_stream_push": (_i32, [_vp, _vp, _i64, _P(bm_fit_report)]),
    "bm_fit_host": (_i32, [_P(bm_config), _vp, _i32, _vp, _vp, _vp, _P(_dbl),
                           _P(bm_fit_report)]),
    "bm_draw_chunk": (_i32, [_i64, _i64, _u64, _i64, _vp, _vp]),
    "bm_gather": (_i32, [_vp, _i64, _i32, _vp, _i64, _vp, _vp]),
    "bm_kpp_reseed": (_i32, [_vp, _i64, _i32, _i32, _vp, _vp, _u64, _i64, _i32, _vp]),
    "bm_lloyd": (_i32, [_vp, _i64, _i32, _i32, _vp, _vp, _i32, _dbl, _P(_dbl),
                        _P(_i32), _vp]),
    "bm_assign_rows": (_i32, [_vp, _i64, _i32, _vp, _vp, _i32, _vp, _vp, _P(_dbl), _vp]),
    "bm_assign_rows_prec": (_i32, [_vp, _i64, _i32, _vp, _vp, _i32, _i32, _vp, _vp,
                                   _P(_dbl), _P(ctypes.c_uint64), _vp]),
    "bm_assign_rows_noalloc": (_i32, [_vp, _i64, _i32, _vp, _vp, _i32, _vp, _vp,
                                      _P(_dbl), _vp]),
    "bm_selftest_wait_timeout": (_i32, [_i32, _vp]),
    "bm_sync_late_reads": (_u64, []),
    "bm_tile_bench": (_i32, [_i32, _i32, _i32, _i32, _i32, _P(_dbl), _P(_u64), _P(_i32),
                             _P(_i32), _vp]),
    "bm_server_create": (_i32, [_P(bm_server_config), _P(_vp)]),
    "bm_server_destroy": (_i32, [_vp]),
    "bm_submit": (_i32, [_vp, _P(bm_job), _P(ctypes.c_uint64)]),
    "bm_wait": (_i32, [_vp, ctypes.c_uint64, _dbl, _P(bm_job_result)]),
    "bm_server_stats_get": (_i32, [_vp, _P(bm_server_stats_t)]),
    "bm_group_create": (_i32, [_P(bm_group_problem), _i32, _i32, _dbl, _i32, _vp, _P(_vp)]),
    "bm_group_run": (_i32, [_vp, _P(bm_group_result), _P(_i32)]),
    "bm_group_info": (_i32, [_vp, _P(_i32), _P(_i32), _P(_i64)]),
    "bm_group_destroy": (_i32, [_vp]),
    "bm_group_set_tiles": (_i32, [_vp, _i32]),
    "bm_group_tiles": (_i32, [_vp, _P(_i32)]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):            # numpy array (host memory)
        return x.ctypes.data
    raise TypeError("expected an address or an object with data_ptr(): %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return getattr(s, "cuda_stream")


def _check(status, where):
    if status != BM_OK:
        raise BigMeansError(status, where)


def bm_status_string(status):
    return _lib.bm_status_string(int(status)).decode()


def bm_config_default(**overrides):
    cfg = bm_config()
    _lib.bm_config_default(ctypes.byref(cfg))
    for key, val in overrides.items():
        setattr(cfg, key, val)
    return cfg


# The native side borrows the memory behind the pointers it is given (a
# context's dataset, a group's problems, a queued job's buffers).  The objects
# that own that memory are kept referenced here, by handle, until the handle
# is destroyed or the job ends, so a temporary tensor passed in is not freed
# (and its memory reused by the caching allocator) while kernels still read it.
_held = {}
_held_ended = set()   # jobs whose end came before their submit returned
_held_lock = threading.Lock()


def _hold(key, *objs):
    with _held_lock:
        if key in _held_ended:
            _held_ended.discard(key)
        else:
            _held[key] = objs


def _release(key, ended=False):
    with _held_lock:
        if _held.pop(key, None) is None and ended:
            _held_ended.add(key)


def bm_create(cfg, X_dev, stream=None):
    ctx = _vp()
    _check(_lib.bm_create(ctypes.byref(cfg), _ptr(X_dev), _stream(stream),
                          ctypes.byref(ctx)), "bm_create")
    _hold(("ctx", ctx.value), X_dev)
    return ctx.value


def bm_destroy(ctx):
    try:
        _check(_lib.bm_destroy(ctx), "bm_destroy")
    finally:
        _release(("ctx", ctx))


def bm_reset(ctx):
    _check(_lib.bm_reset(ctx), "bm_reset")


def bm_fit_chunk(ctx, chunks):
    rep = bm_fit_report()
    _check(_lib.bm_fit_chunk(ctx, int(chunks), ctypes.byref(rep)), "bm_fit_chunk")
    return rep.as_dict()


def bm_assign(ctx, labels_dev=None):
    sse = _dbl()
    _check(_lib.bm_assign(ctx, _ptr(labels_dev), ctypes.byref(sse)), "bm_assign")
    return sse.value


def bm_stream_create(cfg, stream=None):
    """A streaming context (no dataset): portions pushed with bm_stream_push."""
    ctx = _vp()
    _check(_lib.bm_stream_create(ctypes.byref(cfg), _stream(stream), ctypes.byref(ctx)),
           "bm_stream_create")
    return ctx.value


def bm_stream_push(ctx, P_dev, rows):
    """One chunk on the pushed rows (the sample); returns the report."""
    rep = bm_fit_report()
    _check(_lib.bm_stream_push(ctx, _ptr(P_dev), int(rows), ctypes.byref(rep)),
           "bm_stream_push")
    return rep.as_dict()


BM_WORKERS_COMPETITIVE, BM_WORKERS_COLLECTIVE = 0, 1


def bm_fit_workers(ctx, workers, rounds, mode=BM_WORKERS_COLLECTIVE):
    """The paper's parallel modes: `workers` concurrent workers, `rounds` rounds."""
    rep = bm_fit_report()
    _check(_lib.bm_fit_workers(ctx, int(workers), int(rounds), int(mode), ctypes.byref(rep)),
           "bm_fit_workers")
    return rep.as_dict()


def bm_polish(ctx, max_iter=300, tol=1e-4):
    """Full-data Lloyd from the incumbent; returns (f, iterations)."""
    f = _dbl()
    it = _i32()
    _check(_lib.bm_polish(ctx, int(max_iter), float(tol), ctypes.byref(f), ctypes.byref(it)),
           "bm_polish")
    return f.value, it.value


def bm_objective(ctx, C_out_host=None, mask_out_host=None):
    f = _dbl()
    _check(_lib.bm_objective(ctx, ctypes.byref(f), _ptr(C_out_host),
                             _ptr(mask_out_host)), "bm_objective")
    return f.value


def bm_get_state(ctx, C_host, mask_host):
    f = _dbl()
    t = _i64()
    _check(_lib.bm_get_state(ctx, _ptr(C_host), _ptr(mask_host), ctypes.byref(f),
                             ctypes.byref(t)), "bm_get_state")
    return f.value, t.value


def bm_set_state(ctx, C_host, mask_host, f_opt, chunk_counter):
    _check(_lib.bm_set_state(ctx, _ptr(C_host), _ptr(mask_host), float(f_opt),
                             int(chunk_counter)), "bm_set_state")


PHASES = ("setup", "gather", "kmeanspp", "lloyd_own_rows", "lloyd_barrier1",
          "lloyd_reduce", "lloyd_barrier2", "keep", "own_assign", "own_sort",
          "own_sums")


def bm_trace(ctx):
    """Cumulative device time per chunk phase, in ms, keyed by PHASES."""
    buf = (_dbl * len(PHASES))()
    _check(_lib.bm_trace(ctx, buf, len(PHASES)), "bm_trace")
    return {p: buf[i] / 1e6 for i, p in enumerate(PHASES)}


def bm_fit_host(cfg, X_host, chunks, C_out_host=None, mask_out_host=None,
                labels_out_host=None):
    sse = _dbl()
    rep = bm_fit_report()
    _check(_lib.bm_fit_host(ctypes.byref(cfg), _ptr(X_host), int(chunks),
                            _ptr(C_out_host), _ptr(mask_out_host),
                            _ptr(labels_out_host), ctypes.byref(sse),
                            ctypes.byref(rep)), "bm_fit_host")
    return sse.value, rep.as_dict()


def bm_draw_chunk(m, s, seed, t, idx_dev, stream=None):
    _check(_lib.bm_draw_chunk(int(m), int(s), int(seed), int(t), _ptr(idx_dev),
                              _stream(stream)), "bm_draw_chunk")


def bm_gather(X_dev, m, n, idx_dev, s, P_dev, stream=None):
    _check(_lib.bm_gather(_ptr(X_dev), int(m), int(n), _ptr(idx_dev), int(s),
                          _ptr(P_dev), _stream(stream)), "bm_gather")


def bm_kpp_reseed(P_dev, s, n, k, C_dev, mask_dev, seed, t, trials=3, stream=None):
    _check(_lib.bm_kpp_reseed(_ptr(P_dev), int(s), int(n), int(k), _ptr(C_dev),
                              _ptr(mask_dev), int(seed), int(t), int(trials),
                              _stream(stream)), "bm_kpp_reseed")


def bm_lloyd(P_dev, s, n, k, C_dev, mask_dev, max_iter=300, tol=1e-4, stream=None):
    f = _dbl()
    it = _i32()
    _check(_lib.bm_lloyd(_ptr(P_dev), int(s), int(n), int(k), _ptr(C_dev),
                         _ptr(mask_dev), int(max_iter), float(tol), ctypes.byref(f),
                         ctypes.byref(it), _stream(stream)), "bm_lloyd")
    return f.value, it.value


def bm_group_create(problems, max_iter=300, tol=1e-4, balance=True, stream=None):
    """problems: sequence of dicts with P (s x n device rows), s, n, k, C (k x n
    device centroids, the start), mask (k device uint8) and optionally labels
    (s device int32).  Returns a group handle."""
    arr = (bm_group_problem * len(problems))()
    for i, q in enumerate(problems):
        arr[i] = bm_group_problem(_ptr(q["P"]), int(q["s"]), int(q["n"]), int(q["k"]),
                                  _ptr(q["C"]), _ptr(q["mask"]), _ptr(q.get("labels")))
    out = _vp()
    _check(_lib.bm_group_create(arr, len(problems), int(max_iter), float(tol),
                                1 if balance else 0, _stream(stream), ctypes.byref(out)),
           "bm_group_create")
    _hold(("group", out.value), *[(q["P"], q["C"], q["mask"], q.get("labels"))
                                  for q in problems])
    return out.value


def bm_group_run(group, count):
    """Runs the group to convergence; returns (list of result dicts, steps)."""
    res = (bm_group_result * count)()
    steps = _i32()
    _check(_lib.bm_group_run(group, res, ctypes.byref(steps)), "bm_group_run")
    return [r.as_dict() for r in res], steps.value


def bm_group_info(group):
    grid, segs, smem = _i32(), _i32(), _i64()
    _check(_lib.bm_group_info(group, ctypes.byref(grid), ctypes.byref(segs),
                              ctypes.byref(smem)), "bm_group_info")
    return {"grid": grid.value, "segments": segs.value, "smem": smem.value}


def bm_group_set_tiles(group, mode):
    """0: autotune the tile shape per (n, k); 1: a lane per centroid; 2: four
    lanes per row where k <= 16."""
    _check(_lib.bm_group_set_tiles(group, int(mode)), "bm_group_set_tiles")


def bm_group_tiles(group, count):
    """The tile shape of each problem after a run (0 or 1)."""
    buf = (_i32 * count)()
    _check(_lib.bm_group_tiles(group, buf), "bm_group_tiles")
    return [int(v) for v in buf]


def bm_group_destroy(group):
    try:
        _check(_lib.bm_group_destroy(group), "bm_group_destroy")
    finally:
        _release(("group", group))


def bm_assign_rows(X_dev, m, n, C_dev, mask_dev, k, labels_dev=None, dmin_dev=None,
                   stream=None):
    sse = _dbl()
    _check(_lib.bm_assign_rows(_ptr(X_dev), int(m), int(n), _ptr(C_dev),
                               _ptr(mask_dev), int(k), _ptr(labels_dev),
                               _ptr(dmin_dev), ctypes.byref(sse), _stream(stream)),
           "bm_assign_rows")
    return sse.value


def bm_assign_rows_prec(X_dev, m, n, C_dev, mask_dev, k, precision, labels_dev=None,
                        dmin_dev=None, stream=None):
    """Returns (sse, rescored rows)."""
    sse = _dbl()
    resc = ctypes.c_uint64()
    _check(_lib.bm_assign_rows_prec(_ptr(X_dev), int(m), int(n), _ptr(C_dev),
                                    _ptr(mask_dev), int(k), int(precision),
                                    _ptr(labels_dev), _ptr(dmin_dev), ctypes.byref(sse),
                                    ctypes.byref(resc), _stream(stream)),
           "bm_assign_rows_prec")
    return sse.value, resc.value


def bm_assign_rows_noalloc(X_dev, m, n, C_dev, mask_dev, k, labels_dev=None,
                           dmin_dev=None, stream=None):
    """bm_assign_rows without device allocation (scratch inside the library)."""
    sse = _dbl()
    _check(_lib.bm_assign_rows_noalloc(_ptr(X_dev), int(m), int(n), _ptr(C_dev),
                                       _ptr(mask_dev), int(k), _ptr(labels_dev),
                                       _ptr(dmin_dev), ctypes.byref(sse),
                                       _stream(stream)),
           "bm_assign_rows_noalloc")
    return sse.value


def bm_selftest_wait_timeout(timeout_ms=100, stream=None):
    """Status of one grid-barrier wait that runs out (BM_ETIMEOUT expected)."""
    return _lib.bm_selftest_wait_timeout(int(timeout_ms), _stream(stream))


def bm_tile_bench(n, k, planes=1, steps=4096, epilogue=True, stream=None):
    """The distance-tile pipeline with resident operands: dict(ms, checksum,
    grid, tiles)."""
    ms, cks, grid, tiles = _dbl(), _u64(), _i32(), _i32()
    _check(_lib.bm_tile_bench(int(n), int(k), int(planes), int(steps), 1 if epilogue else 0,
                              ctypes.byref(ms), ctypes.byref(cks), ctypes.byref(grid),
                              ctypes.byref(tiles), _stream(stream)), "bm_tile_bench")
    return {"ms": ms.value, "checksum": cks.value, "grid": grid.value, "tiles": tiles.value}


def bm_sync_late_reads():
    """K-means++ exchange values found not yet published after their grid
    barrier (each waited for), summed over the process so far."""
    return int(_lib.bm_sync_late_reads())


# ------------------------------------------------------------------ serving
def bm_server_create(workers=2, memory_budget=0, max_queue=256, job_ctas=0):
    cfg = bm_server_config(int(workers), int(memory_budget), int(max_queue), int(job_ctas))
    sv = _vp()
    _check(_lib.bm_server_create(ctypes.byref(cfg), ctypes.byref(sv)), "bm_server_create")
    return sv.value


def bm_server_destroy(server):
    try:
        _check(_lib.bm_server_destroy(server), "bm_server_destroy")
    finally:
        with _held_lock:
            for key in [q for q in _held if q[0] == "job" and q[1] == server]:
                del _held[key]
            _held_ended.difference_update(
                [q for q in _held_ended if q[0] == "job" and q[1] == server])


def bm_submit(server, cfg, X_dev, chunks, labels_dev=None, C_out_host=None,
              mask_out_host=None, callback=None):
    """Admits a job; returns its ticket.  callback(ticket, result_dict) runs on
    a worker thread when the job ends.  The job's buffers (and the callback)
    stay referenced until the job's result is taken by bm_wait or handed to
    the callback."""
    job = bm_job()
    job.cfg = cfg
    job.X_dev = _ptr(X_dev)
    job.chunks = int(chunks)
    job.labels_dev = _ptr(labels_dev)
    job.C_out_host = _ptr(C_out_host)
    job.mask_out_host = _ptr(mask_out_host)
    holder = None
    if callback is not None:
        def _cb(ticket, res, user, _f=callback):
            try:
                _f(int(ticket), res.contents.as_dict())
            finally:
                _release(("job", server, int(ticket)), ended=True)
        holder = bm_job_callback(_cb)
        job.callback = holder
    ticket = ctypes.c_uint64()
    _check(_lib.bm_submit(server, ctypes.byref(job), ctypes.byref(ticket)), "bm_submit")
    _hold(("job", server, ticket.value), holder, X_dev, labels_dev, C_out_host, mask_out_host)
    return ticket.value


def bm_wait(server, ticket, timeout=-1.0):
    """The job's result as a dict, or None if it is still pending after
    `timeout` seconds (< 0: no limit)."""
    res = bm_job_result()
    st = _lib.bm_wait(server, ctypes.c_uint64(ticket), float(timeout), ctypes.byref(res))
    if st == BM_ETIMEOUT:
        return None
    _check(st, "bm_wait")
    _release(("job", server, int(ticket)))
    return res.as_dict()


def bm_server_stats(server):
    out = bm_server_stats_t()
    _check(_lib.bm_server_stats_get(server, ctypes.byref(out)), "bm_server_stats_get")
    return out.as_dict()
