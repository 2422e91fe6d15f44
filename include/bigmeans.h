/*
 * bigmeans.h -- C ABI of the GB300 Big-means library (libbigmeans.so).
 *
 * Big-means (Mussabayev, Mladenovic, Mussabayev, Jarboui, "How to Use
 * K-means for Big Data Clustering?", arXiv 2204.07485) solves the minimum
 * sum-of-squares clustering problem (Sec. 1, Eq. 1): given m points X in R^n
 * and k, find centroids C minimising f(C, X) = sum_i min_j ||x_i - c_j||^2.
 * Alg. 1 repeatedly draws a uniform sample P of s points (Sec. 3.1, Eq. 2;
 * Sec. 3.5), reinitialises the degenerate centroids of the incumbent with
 * K-means++ (Sec. 3.3), runs K-means on P (Sec. 2), keeps the result if its
 * sample objective beats the incumbent's (Alg. 1, Sec. 3.2), and finally
 * assigns every point of X to its nearest centroid (Sec. 3.4).
 *
 * Conventions for every entry point
 *   - Matrices are row-major float32: X is m x n, P is s x n, C is k x n.
 *   - "_dev" pointers are CUDA device pointers, "_host" pointers host memory.
 *     Device buffers passed in are borrowed: the caller owns them and must
 *     keep them alive for the duration of the call (X_dev: for the whole
 *     lifetime of the context that borrows it).
 *   - A centroid mask holds one byte per centroid: 1 = live, 0 = degenerate
 *     (empty or uninitialised, Alg. 1 / Sec. 3.3).  The coordinates of a
 *     degenerate centroid are never read.
 *   - stream is a cudaStream_t (NULL = legacy default stream).
 *   - Every call returns a bm_status and never aborts the process.  Invalid
 *     shapes return BM_EINVAL (k < 1, n < 1, s < 1, s > m, k > s, m or s
 *     beyond 2^31 - 1); CUDA failures return BM_ECUDA; a device-side wait
 *     that exceeds its bound returns BM_ETIMEOUT and leaves the context
 *     usable after bm_reset.
 *   - Results are a pure function of (X, configuration, seed) on a given
 *     device: reductions have a fixed shape and order (no float atomics).
 *   - Random draws follow Philox4x64-10 (Salmon et al., SC'11) with
 *     key (seed, 0) and counter (i / 4, round, chunk t, purpose), word i % 4.
 */
#ifndef BIGMEANS_H
#define BIGMEANS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bm_status {
  BM_OK = 0,
  BM_EINVAL = 1,        /* invalid argument or shape                         */
  BM_ENOMEM = 2,        /* device allocation or admission failed              */
  BM_ECUDA = 3,         /* a CUDA runtime call failed                         */
  BM_ETIMEOUT = 4,      /* a bounded device-side wait gave up                 */
  BM_EBUSY = 5,         /* server full / resource in use                      */
  BM_ECANCELLED = 6,    /* job cancelled before completion                   */
  BM_EUNSUPPORTED = 7,  /* shape outside what the library's kernels cover    */
  BM_EGUARD = 8         /* debug builds only (BM_DEBUG_GUARDS): a device index
                           guard found an access outside its buffer and
                           skipped it                                        */
} bm_status;

typedef enum bm_precision {
  BM_FP32 = 0,          /* FP32 distances throughout                          */
  BM_BF16_RESCORE = 1,  /* BF16 tensor-core distances, FP32 rescore of ties   */
  BM_FP8_RESCORE = 2,   /* FP8 E4M3 tensor-core distances (rows and centroids
                           scaled by powers of two), FP32 rescore             */
  BM_BF16X3_RESCORE = 3 /* split BF16 (hi*hi + hi*lo + lo*hi) tensor-core
                           distances, FP32 rescore of the few remaining ties  */
} bm_precision;

/* Reinitialisation of degenerate centroids at the start of a chunk. */
typedef enum bm_init {
  BM_INIT_KMEANSPP = 0, /* K-means++ with kpp_trials candidates, lowest potential
                           (the paper's choice, Sec. 3.3 and 5)               */
  BM_INIT_FORGY = 1     /* Forgy (Sec. 2): each degenerate slot j takes the sample
                           row floor(u_j * s), u_j its first K-means++ uniform;
                           no distance evaluations                           */
} bm_init;

/* What Lloyd does with a live centroid that loses all its members (the paper
 * leaves the empty-cluster rule open as an interchangeable ingredient). */
typedef enum bm_empty {
  BM_EMPTY_DEGENERATE = 0, /* it becomes degenerate: out of the rest of the
                              chunk, reseeded at the next chunk (Sec. 3.3)    */
  BM_EMPTY_KEEP = 1        /* it keeps its position and stays live, so it can
                              win rows again at a later step                 */
} bm_empty;

/* Parameters of one Big-means job (Alg. 1 inputs X, k, s and the stop rule). */
typedef struct bm_config {
  int64_t m;            /* number of points                                    */
  int32_t n;            /* dimension                                           */
  int32_t k;            /* number of clusters                                  */
  int64_t s;            /* sample (chunk) size, 1 <= s <= m, k <= s            */
  int32_t max_iter;     /* Lloyd update-step cap per chunk (Sec. 5: 300)       */
  double tol;           /* Lloyd relative-improvement stop (Sec. 5: 1e-4)      */
  int32_t kpp_trials;   /* K-means++ candidates per new centre (Sec. 5: 3)     */
  uint64_t seed;        /* Philox key                                          */
  int32_t precision;    /* bm_precision                                        */
  double time_budget_s; /* bm_fit_chunk(chunks = 0) runs until this elapses    */
  int32_t graphs;       /* 1: bm_fit_chunk(chunks > 0) records its launches in
                           a CUDA graph once per launch state and replays it;
                           0: launches one kernel at a time                    */
  int32_t trace;        /* 1: the chunk kernel times its phases (bm_trace);
                           costs a timer read per phase on CTA 0               */
  int32_t max_ctas;     /* > 0: at most this many CTAs per chunk launch (and
                           SMs' worth of final-assignment CTAs), leaving the
                           other SMs to concurrent jobs; 0: no cap             */
  int32_t init;         /* bm_init: how degenerate centroids are reinitialised */
  int32_t empty;        /* bm_empty: Lloyd's rule for a centroid without members
                           (grouped problems and bm_lloyd use the default)     */
} bm_config;

/* What one bm_fit_chunk call did. */
typedef struct bm_fit_report {
  int64_t chunks;        /* chunks processed by this call                      */
  int64_t accepted;      /* of which replaced the incumbent (Alg. 1)           */
  int64_t lloyd_iters;   /* Lloyd update steps summed over those chunks        */
  int64_t n_d;           /* distance evaluations, cumulative for the context   */
  int64_t chunk_counter; /* index t of the next chunk                          */
  double f_opt;          /* incumbent sample objective after the call          */
  double seconds;        /* host wall time of the call                         */
  int64_t host_gathers;  /* CTA gathers of this call made while part of X
                            was still only in host memory (bm_fit_host, while
                            its copy of X is in flight); 0 otherwise          */
} bm_fit_report;

typedef struct bm_ctx bm_ctx;

/* Fills *cfg with the paper's defaults (max_iter 300, tol 1e-4, 3 trials,
 * FP32, seed 0, K-means++ reinitialisation), graph replay on, phase tracing
 * off, no CTA cap, and zero sizes. */
void bm_config_default(bm_config* cfg);

/* Human-readable name of a status code (static string). */
const char* bm_status_string(int32_t status);

/* Creates a Big-means context for the dataset X_dev (m x n, borrowed: it
 * must stay valid and unchanged until bm_destroy) on the current CUDA device.  Allocates all device state (sample, centroids,
 * partial sums) once.  The incumbent starts with every centroid degenerate
 * and f_opt = +inf (Alg. 1).  stream: the stream all work is queued on. */
bm_status bm_create(const bm_config* cfg, const float* X_dev, void* stream,
                    bm_ctx** out);

/* Releases the context (synchronises its stream first).  NULL is a no-op. */
bm_status bm_destroy(bm_ctx* ctx);

/* Resets the incumbent to all-degenerate, f_opt = +inf, chunk counter 0,
 * n_d = 0, and clears any error left by a failed launch. */
bm_status bm_reset(bm_ctx* ctx);

/* Runs Alg. 1's loop body for `chunks` consecutive chunks t, t+1, ...:
 * draw sample t, gather P, K-means++ reseed of degenerate centroids, Lloyd on
 * P, keep-the-best.  chunks = 0 runs chunks until cfg.time_budget_s of wall
 * time has elapsed (the paper's CPU-time stop condition, Sec. 5).  Blocks
 * until the work is done; `out` (may be NULL) receives the report.  With
 * cfg.graphs = 1 the launches of a call are recorded once per (first chunk,
 * chunks, launch parity, sample-plan window) and replayed as one CUDA graph
 * afterwards (a context keeps the four most recent); results are identical
 * either way. */
bm_status bm_fit_chunk(bm_ctx* ctx, int32_t chunks, bm_fit_report* out);

/* Final step of Alg. 1: labels_dev[i] (int32, m entries, caller-owned device
 * memory; may be NULL to skip labels) = nearest live incumbent centroid of
 * x_i (lowest index on ties); *sse_out (host, may be NULL) = f(C, X)
 * accumulated in float64.  With a tensor-core precision form (BM_BF16_RESCORE,
 * BM_BF16X3_RESCORE, BM_FP8_RESCORE) the distances run on the tensor cores in
 * that arithmetic with exact FP32 rescoring (see bm_assign_rows_prec); the
 * chunks of a context (rows wider than 32 features) screen with BF16
 * products in BM_BF16_RESCORE, E4M3 products in BM_FP8_RESCORE (rows scaled
 * per row, centroids by one power of two per chunk) and split BF16 products
 * otherwise (labels and distances are those of FP32 either way).  Blocks
 * until done. */
bm_status bm_assign(bm_ctx* ctx, int32_t* labels_dev, double* sse_out);

/* Streaming (stream processing of newly arriving data portions, Sec. 1 and
 * 7): a context without a resident dataset.  cfg.s is the largest portion;
 * cfg.m is ignored.  Each bm_stream_push treats the pushed rows (device,
 * rows x n row-major, k <= rows <= cfg.s, borrowed for the call) as the next
 * chunk's sample: K-means++ (or Forgy) reseed, Lloyd, keep-the-best against
 * the incumbent, with the chunk counter advancing by one.  bm_get_state /
 * bm_set_state / bm_objective / bm_reset work as for any context;
 * bm_fit_chunk, bm_assign, bm_polish and bm_fit_workers need a dataset and
 * return BM_EINVAL (assign other data with bm_assign_rows and the incumbent).
 * Release with bm_destroy. */
bm_status bm_stream_create(const bm_config* cfg, void* stream, bm_ctx** out);
bm_status bm_stream_push(bm_ctx* ctx, const float* P_dev, int64_t rows, bm_fit_report* out);

/* Parallel Big-means workers on one GPU (the paper's parallelisation modes
 * 2 and 3, Sec. 3.5).  `workers` worker contexts run side by side on their own
 * streams (each capped at cfg.max_ctas CTAs, default SMs / workers); in round
 * r worker w processes chunk t + r * workers + w of this context's chunk
 * sequence (its own sample).  BM_WORKERS_COMPETITIVE: each worker keeps its
 * own incumbent, starting from this context's, and after the last round the
 * best one (lowest f_opt, lowest worker on ties) replaces this context's when
 * strictly better.  BM_WORKERS_COLLECTIVE: every round starts all workers
 * from this context's incumbent, and the best of their results (same order)
 * replaces it when strictly better.  The chunk counter advances by
 * rounds * workers.  `out` (may be NULL) sums the workers' chunks, accepted
 * chunks and Lloyd steps.  Blocks until done. */
enum { BM_WORKERS_COMPETITIVE = 0, BM_WORKERS_COLLECTIVE = 1 };
bm_status bm_fit_workers(bm_ctx* ctx, int32_t workers, int32_t rounds, int32_t mode,
                         bm_fit_report* out);

/* Full-data Lloyd polish (the further SSE reduction Sec. 3.4 suggests after
 * Big-means): Lloyd iterations on all of X starting from the incumbent, with
 * the chunks' stop rule (after an assignment: stop if f = 0, or it > 0 and
 * f_prev - f <= tol * f_prev, or it = max_iter; centroids left without
 * members become degenerate).  The resulting centroids and mask replace the
 * incumbent; f_opt keeps its sample value.  *f_out (may be NULL) = f(C, X) of
 * the last assignment (the returned centroids), *iters_out = update steps.
 * Each iteration streams X twice (assignment, then the update's per-CTA
 * partial sums over fixed row ranges); every sum has a fixed order.  Needs
 * a live incumbent (else BM_EINVAL).  Blocks until done. */
bm_status bm_polish(bm_ctx* ctx, int32_t max_iter, double tol, double* f_out,
                    int32_t* iters_out);

/* Reads the incumbent: f_opt (its sample objective), C (k x n, host) and the
 * mask (k bytes, host).  Any output may be NULL. */
bm_status bm_objective(bm_ctx* ctx, double* f_opt_out, float* C_out_host,
                       uint8_t* mask_out_host);

/* Checkpoint / resume of the whole Alg. 1 state: incumbent C (k x n host),
 * mask (k host), f_opt and the next chunk index.  Restoring a saved state
 * and continuing reproduces an uninterrupted run bit for bit. */
bm_status bm_get_state(bm_ctx* ctx, float* C_host, uint8_t* mask_host,
                       double* f_opt, int64_t* chunk_counter);
bm_status bm_set_state(bm_ctx* ctx, const float* C_host,
                       const uint8_t* mask_host, double f_opt,
                       int64_t chunk_counter);

/* Tracing: cumulative device time (ns) of the chunk phases since bm_create
 * or bm_reset, as seen by CTA 0 between its phase boundaries: [0] set-up,
 * [1] gather, [2] K-means++ reseed, [3] Lloyd assignment + partial sums of
 * CTA 0's rows, [4] wait at the first Lloyd grid barrier, [5] cross-CTA
 * reduction + centroid update, [6] wait at the second barrier + reload,
 * [7] keep-the-best; [8], [9], [10] split [3] -- row-in-register kernels:
 * the assignment, the stable sort of the rows by label, and the per-centroid
 * sums into the partial sums; tensor-core kernel: the tensor-core candidate
 * pass, the multi-candidate rows plus the label sort, and the staged exact
 * sweep.
 * ns_out receives min(count, 11) values.  The times are collected only by
 * contexts created with cfg.trace = 1 (each timer read sits on CTA 0's path
 * to the next grid barrier, so tracing slows the run slightly); otherwise
 * they stay zero. */
bm_status bm_trace(bm_ctx* ctx, double* ns_out, int32_t count);

/* One-call job on HOST memory: copies X_host (m x n) to the device, runs
 * `chunks` chunks and the final assignment, and copies back C (k x n),
 * mask (k), labels (m) and f(C, X).  Outputs may be NULL.  Uses its own
 * stream; its device memory comes from a stream-ordered pool per device that
 * the library keeps (with the freed blocks, for the next call) until the
 * process exits.  When X_host is pinned or registered host memory (readable
 * by the GPU in place), the copy runs on a second stream, in 32 interleaved
 * pieces (X cut into blocks of a power-of-two number of rows, at most
 * m / 4096; piece p holds every 32nd block from block p), while the chunks
 * start at once: a CTA gathers each sample row from the device copy when the
 * row's piece has landed and from host memory otherwise (the same bytes, so
 * the results are those of the copied path); the final assignment waits for
 * the copy.  report->host_gathers counts the CTA gathers made before the
 * last piece landed.
 * X_host must stay unchanged during the call. */
bm_status bm_fit_host(const bm_config* cfg, const float* X_host,
                      int32_t chunks, float* C_out_host,
                      uint8_t* mask_out_host, int32_t* labels_out_host,
                      double* sse_out, bm_fit_report* report);

/* ---------------------------------------------------------------------
 * Step-level entry points: each runs one step of the hot path on caller
 * buffers, on `stream`, and blocks until done.  Each call allocates its
 * scratch (partial sums, barrier counters) on the current device and frees
 * it before returning; calls from several host threads serialise on a lock.
 * ------------------------------------------------------------------- */

/* Sample draw of chunk t (Sec. 3.1, Eq. 2; Sec. 3.5): writes the s sorted,
 * distinct row indices of the uniform sample to idx_dev (int32, s entries).
 * Round r draws (count - |S|) Philox values (purpose 0) mapped to [0, m) by
 * the high word of a 64x64 product and adds them to S; for 2s > m the m - s
 * rows to leave out are drawn instead and the sample is their complement. */
bm_status bm_draw_chunk(int64_t m, int64_t s, uint64_t seed, int64_t t,
                        int32_t* idx_dev, void* stream);

/* P = X[idx] (Alg. 1: "P <- uniform random sample"): P_dev is s x n. */
bm_status bm_gather(const float* X_dev, int64_t m, int32_t n,
                    const int32_t* idx_dev, int64_t s, float* P_dev,
                    void* stream);

/* K-means++ reseed (Sec. 2; Sec. 3.3; three candidates, Sec. 5) of every
 * degenerate centroid of (C_dev, mask_dev) (k x n and k bytes, updated in
 * place) on the sample P_dev (s x n), in ascending slot order, with the
 * uniforms of chunk t (purposes 1 and 2 of the Philox stream). */
bm_status bm_kpp_reseed(const float* P_dev, int64_t s, int32_t n, int32_t k,
                        float* C_dev, uint8_t* mask_dev, uint64_t seed,
                        int64_t t, int32_t trials, void* stream);

/* K-means (Lloyd) on P_dev from (C_dev, mask_dev) (Sec. 2; stop rule Sec. 5):
 * updates C and the mask in place (clusters that empty become degenerate),
 * *f_out (host) = f(C'', P) in float64, *iters_out (host) = update steps. */
bm_status bm_lloyd(const float* P_dev, int64_t s, int32_t n, int32_t k,
                   float* C_dev, uint8_t* mask_dev, int32_t max_iter,
                   double tol, double* f_out, int32_t* iters_out,
                   void* stream);

/* Nearest-centroid assignment of arbitrary rows (Alg. 1's final step,
 * Sec. 3.4): labels_dev[i] (int32, may be NULL) = nearest live centroid,
 * dmin_dev[i] (float32, may be NULL) = its squared distance, *sse_out (host,
 * may be NULL) = sum of those distances accumulated in float64. */
bm_status bm_assign_rows(const float* X_dev, int64_t m, int32_t n,
                         const float* C_dev, const uint8_t* mask_dev,
                         int32_t k, int32_t* labels_dev, float* dmin_dev,
                         double* sse_out, void* stream);

/* bm_assign_rows with a choice of distance arithmetic.  BM_FP32 is
 * bm_assign_rows.  BM_BF16_RESCORE computes the dot products x.c_j on the
 * tensor cores in BF16 with FP32 accumulation, bounds the error of every
 * resulting distance, and rescores in exact FP32 every row for which more
 * than one centroid lies within the bounds; labels and distances equal those
 * of the FP32 arithmetic.  BM_BF16X3_RESCORE does the same with split BF16
 * products (tighter bounds, fewer rescored rows); BM_FP8_RESCORE with E4M3
 * products of rows and centroids each scaled by a power of two into
 * [128, 256) (looser bounds, more rescored rows).  *rescored_out (host, may
 * be NULL) receives the number of rescored rows.  k <= 128.  Blocks until
 * done. */
bm_status bm_assign_rows_prec(const float* X_dev, int64_t m, int32_t n,
                              const float* C_dev, const uint8_t* mask_dev,
                              int32_t k, int32_t precision, int32_t* labels_dev,
                              float* dmin_dev, double* sse_out,
                              uint64_t* rescored_out, void* stream);

/* Allocation-free variant of bm_assign_rows (same arguments, same results
 * within rounding).  The paper has no counterpart: this serves callers that
 * cannot allocate device memory when they need an assignment -- a process
 * that has handed its device memory to its own pool allocator, or a
 * latency-critical loop that cannot afford cudaMalloc / cudaFree, which may
 * synchronise the whole device.  The call allocates nothing: its scratch (one
 * float64 partial per CTA, the last-CTA ticket and the result, 16,640 bytes)
 * is a fixed array inside the library that every GPU loading the library
 * holds until the process exits.  The first call on each device looks up that
 * array's device address (cudaGetSymbolAddress, with the device current).
 * All calls share the one array, and calls that overlapped on the GPU would
 * race on it: so every call holds a lock inside the library from its first
 * use of the array until its result has been read back (the call blocks
 * until its work is done), and calls from several host threads of the
 * process, on one stream or on several, run one after another.  A launch that would need more than 2048
 * CTAs, k > 128, or a centroid table beyond shared memory (where
 * bm_assign_rows would switch to the tensor-core kernel, whose scratch grows
 * with m) returns BM_EUNSUPPORTED. */
bm_status bm_assign_rows_noalloc(const float* X_dev, int64_t m, int32_t n,
                                 const float* C_dev, const uint8_t* mask_dev,
                                 int32_t k, int32_t* labels_dev,
                                 float* dmin_dev, double* sse_out,
                                 void* stream);

/* Failure-detection self-test: runs one wait of the grid barrier that the
 * chunk kernels use between phases, with a participant that never arrives
 * and a limit of timeout_ms (1 .. 2000).  The wait gives up, records the
 * timeout in its status word and returns; the call returns BM_ETIMEOUT (any
 * other status means the bounded wait is broken) and the device stays usable.
 * Nothing faults, traps or hangs.  BM_EINVAL for a limit out of range. */
bm_status bm_selftest_wait_timeout(int32_t timeout_ms, void* stream);

/* Measurement of the distance-tile pipeline alone (the paper has no
 * counterpart; it separates the tensor-core tile design from the data
 * movement around it).  One CTA per SM keeps `tiles` 128-row A tiles of n
 * features (n = 64, 128, 192 or 256) and a block of k centroids (1..128) in
 * shared memory as BF16 (planes = 1) or split BF16 (planes = 2) operands of
 * small integers, loaded once; then runs `steps` tile steps, each the
 * tcgen05.mma of one tile into one of two TMEM accumulators and, with
 * epilogue != 0, the candidate epilogue of the chunk kernel on it (per row:
 * the minimum of ||c_j||^2 - 2 x.c_j, then the count of columns within 0.5
 * of it), the MMA of the next step overlapping the epilogue.  *ms_out = the
 * launch's time (CUDA events on `stream`); *checksum_out = the sum over CTAs,
 * steps and rows of argmin + 1024 x count (exact: the operands are integers);
 * *grid_out = CTAs; *tiles_out = resident tiles (step s uses tile s mod
 * tiles).  A tile's A operand is tb_a(tile, r, f) = ((7 r + 3 f + 5 tile) mod
 * 5) - 2 and centroid j's feature f is ((11 j + 13 f) mod 7) - 3.  Allocates
 * 16 bytes of scratch; blocks until done.  BM_EINVAL for shapes outside the
 * ranges above. */
bm_status bm_tile_bench(int32_t n, int32_t k, int32_t planes, int32_t steps,
                        int32_t epilogue, double* ms_out, uint64_t* checksum_out,
                        int32_t* grid_out, int32_t* tiles_out, void* stream);

/* Self-check of the K-means++ reseed (Sec. 3.3) across CTAs.  The values the
 * CTAs of a chunk launch hand to each other between grid barriers while they
 * pick a new centre (per-CTA D^2 sums, the candidate rows, the candidates'
 * potentials) each carry a tag of their launch and slot; a reader checks the
 * tag before it uses the value, waits (bounded; BM_ETIMEOUT on expiry) if the
 * value has not been published yet, and counts that event.  Returns the
 * number of such late reads in this process since the library was loaded,
 * summed when the status of each launch is read back (end of bm_fit_chunk,
 * bm_stream_push, bm_fit_workers, bm_fit_host, bm_kpp_reseed, bm_lloyd and
 * the server's jobs).  0 means every exchange found its value published by
 * the time the barrier released the reader.  Thread-safe. */
uint64_t bm_sync_late_reads(void);

/* ------------------------------------------------------------ grouped Lloyd
 * Many independent Lloyd problems (Sec. 2, stop rule of Sec. 5) -- the
 * chunks of many Big-means jobs, say -- advanced together: each Lloyd step
 * of every unfinished problem is one cooperative launch that assigns all
 * their rows, waits at a grid barrier and updates all their centroids (two
 * launches when the grid cannot be co-resident), and a recorded CUDA graph
 * replays the steps.  The rows of all problems are cut into per-CTA ranges
 * of equal cost, so one large problem spreads over many SMs and small ones
 * share an SM; between replays the unfinished problems are cut again over
 * the whole GPU.  Each problem ends where bm_lloyd alone would: the same stop
 * rule, the same degenerate-cluster handling (live centroids that lose every
 * member become degenerate), objectives and centroids equal to rounding
 * (the sums run over a different row partition). */
typedef struct bm_group bm_group;

typedef struct bm_group_problem {
  const float* P_dev;     /* s x n rows, row-major float32, device (borrowed)    */
  int64_t s;              /* rows, >= k                                           */
  int32_t n;              /* features, 1 .. 512                                   */
  int32_t k;              /* centroid slots, 1 .. 128                             */
  float* C_dev;           /* k x n row-major centroids, device: the start on
                             entry to bm_group_run, the result after it          */
  uint8_t* mask_dev;      /* k live flags (1 = live), device, in and out         */
  int32_t* labels_dev;    /* s labels of the last assignment (device, may be NULL) */
} bm_group_problem;

typedef struct bm_group_result {
  double f;               /* objective of the last assignment (float64)          */
  int64_t n_d;            /* point-centroid distance evaluations                  */
  int32_t iters;          /* update steps                                         */
  int32_t live;           /* live centroids at the end                            */
} bm_group_result;

/* Plans a group: validates the problems (BM_EINVAL: NULL buffers, s < k,
 * n < 1, k < 1, count < 1, max_iter < 0, tol < 0; BM_EUNSUPPORTED: k > 128,
 * n > 512, or tables beyond shared memory), partitions their rows over the
 * GPU (balance = 1; balance = 0 gives each problem a single CTA of its own)
 * and allocates the partial results.  The problems' buffers are borrowed
 * until bm_group_destroy.  Work goes to `stream` (NULL: the legacy stream,
 * without graph replay). */
bm_status bm_group_create(const bm_group_problem* problems, int32_t count,
                          int32_t max_iter, double tol, int32_t balance,
                          void* stream, bm_group** out);

/* Runs every problem from its current C and mask to its stop; blocks until
 * done.  results_host (count entries, may be NULL) receives each problem's
 * outcome, *steps_out (may be NULL) the Lloyd steps launched. */
bm_status bm_group_run(bm_group* group, bm_group_result* results_host, int32_t* steps_out);

/* The plan: CTAs of the assignment launch, segments of the partition of all
 * problems, dynamic shared memory. */
bm_status bm_group_info(bm_group* group, int32_t* grid_out, int32_t* segments_out,
                        int64_t* smem_out);

/* Tile shape of the assignment's 64-row tiles: mode 0 (default) lets the
 * group's first run time, for every (n, k) with k <= 16, a lane per centroid
 * against four lanes per row and keep the faster for those problems; mode 1
 * keeps a lane per centroid everywhere; mode 2 takes four lanes per row
 * wherever k <= 16.  The shapes add the same terms in the same order, so the
 * results do not depend on the mode.  The next bm_group_run applies it. */
bm_status bm_group_set_tiles(bm_group* group, int32_t mode);

/* The tile shape each problem uses (count entries, host): 0 = a lane per
 * centroid, 1 = four lanes per row; meaningful after a run. */
bm_status bm_group_tiles(bm_group* group, int32_t* shapes_host);

/* Frees the group (NULL is a no-op). */
bm_status bm_group_destroy(bm_group* group);

/* ------------------------------------------------------------------ serving
 * A job server runs whole Big-means jobs (Alg. 1: `chunks` chunks, then the
 * final assignment) submitted from any thread, several at a time on one GPU.
 * Each worker thread owns a CUDA stream; a job's device state comes from a
 * stream-ordered memory pool the server owns, so jobs allocate and free
 * without synchronising the device.  The paper runs one job at a time; the
 * server adds admission control and request latency on top of the same
 * kernels, and a job's results do not depend on what else is running (every
 * reduction has a fixed order). */
typedef struct bm_server bm_server;

typedef struct bm_server_config {
  int32_t workers;        /* jobs run at once (threads, each with a stream), >= 1 */
  int64_t memory_budget;  /* device bytes the admitted jobs' state may hold at
                             once; 0 = half the device memory free at creation  */
  int32_t max_queue;      /* admitted jobs waiting for a worker (>= 1)          */
  int32_t job_ctas;       /* CTA cap of a job whose cfg.max_ctas is 0 (>= 0;
                             0 = ceil(SMs / 2)).  It does not depend on
                             `workers`, so a job's results are those of the
                             same configuration with max_ctas = this cap run
                             alone, whatever the server's size               */
} bm_server_config;

/* What a finished job produced (and how long it took on the host clock). */
typedef struct bm_job_result {
  int32_t status;         /* bm_status of the job; BM_ECANCELLED if the server
                             shut down before it started                         */
  double sse;             /* f(C, X) of the final assignment, float64            */
  double f_opt;           /* incumbent sample objective                           */
  int64_t lloyd_iters;    /* Lloyd update steps over all chunks                   */
  int64_t accepted;       /* chunks that replaced the incumbent                   */
  double queued_s;        /* submission -> a worker starts it                    */
  double run_s;           /* start -> results ready                              */
  double latency_s;       /* submission -> results ready                         */
} bm_job_result;

typedef void (*bm_job_callback)(uint64_t ticket, const bm_job_result* result, void* user);

/* One job.  X_dev (m x n, device) and the output buffers are borrowed until
 * the job completes; any output may be NULL. */
typedef struct bm_job {
  bm_config cfg;              /* sizes, stop rule, seed, precision (graphs ignored;
                                 max_ctas = 0 means SMs / workers)                 */
  const float* X_dev;
  int32_t chunks;             /* chunks to run, > 0                                */
  int32_t* labels_dev;        /* m labels of the final assignment (device)         */
  float* C_out_host;          /* k x n incumbent centroids (host)                   */
  uint8_t* mask_out_host;     /* k live flags (host)                                */
  bm_job_callback callback;   /* called from a worker thread when the job ends     */
  void* user;
} bm_job;

/* Counters of a server. */
typedef struct bm_server_stats {
  int64_t submitted, completed, failed, cancelled;
  int64_t rejected_busy, rejected_memory;
  int64_t queued, running;
  int64_t memory_in_use, memory_budget;
} bm_server_stats;

/* Starts `workers` worker threads on the current device. */
bm_status bm_server_create(const bm_server_config* cfg, bm_server** out);

/* Stops accepting jobs, cancels the queued ones (their result status is
 * BM_ECANCELLED and their callbacks run), waits for the running ones, joins
 * the workers and frees the pool.  NULL is a no-op. */
bm_status bm_server_destroy(bm_server* server);

/* Admits a job and returns its ticket; thread-safe.  BM_EINVAL: bad
 * arguments or shapes; BM_EUNSUPPORTED: a shape no kernel handles; BM_ENOMEM:
 * the job alone needs more than the memory budget; BM_EBUSY: the queue is
 * full; BM_ECANCELLED: the server is shutting down.  An admitted job waits
 * (first in, first out) until a worker is free and its state fits in what
 * the running jobs leave of the budget. */
bm_status bm_submit(bm_server* server, const bm_job* job, uint64_t* ticket);

/* Waits up to timeout_s seconds (< 0: no limit) for the job's result.
 * BM_ETIMEOUT when it is still pending (the ticket stays valid); BM_OK with
 * *out filled, after which the ticket is gone.  Jobs submitted with a
 * callback hand their result to the callback instead and are gone once it
 * returns; waiting for them returns BM_EINVAL after that.  A bad ticket
 * returns BM_EINVAL. */
bm_status bm_wait(bm_server* server, uint64_t ticket, double timeout_s, bm_job_result* out);

/* Snapshot of the server's counters. */
bm_status bm_server_stats_get(bm_server* server, bm_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* BIGMEANS_H */
