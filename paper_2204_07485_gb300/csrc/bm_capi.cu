// C ABI of the Big-means library: contexts, the chunk driver and the
// step-level entry points.  All compute runs in the kernels of
// bm_kernels.cu; this file sizes buffers, picks a launch shape, queues the
// launches on the caller's stream and reports status.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <atomic>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_internal.h"

namespace bm {

// ------------------------------------------------------------------ plan
// Kernel family and launch shape for one (n, k, s) on the current device.
struct Plan {
  bool tc = false;   // tensor-core chunk kernel (rows wider than 32 features)
  bool generic = false;
  int np = 0;        // register row width of the np path
  int npad = 0;      // row stride of P and C (floats)
  int kpad = 0;      // k rounded up to 32 (generic path)
  int grid = 0;      // CTAs of the chunk kernel
  int R = 0;         // sample rows per CTA
  size_t smem = 0;   // dynamic shared memory of the chunk kernel
  int agrid = 0;     // CTAs of the FP32 assign kernel (0: tensor cores only)
  size_t asmem = 0;
  int tc_kb = 0, tc_n16 = 0, tc_ncols = 0, tc_fb = 0, tc_ns = 0, tc_tpc = 0;
  int tc_planes = 2; // planes of the chunk kernel's screening (1 or 2)
  int tc_fp8 = 0;    // 1: the chunk kernel screens with E4M3 products
  int cap = 0;       // CTA cap of the job (bm_config.max_ctas), 0 = none
};

static constexpr size_t kSmemLimit = 227 * 1024;

static int sm_count() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Tensor-core chunk plan: one CTA per SM (TMEM, grid barrier), at least one
// 128-row tile per CTA, the widest staged feature block that fits.
static bm_status make_plan_tc(int n, int k, long long s, Plan* out, int cap, int planes,
                              bool fp8) {
  if (k > kMaxK || n > 512) return BM_EUNSUPPORTED;
  Plan p;
  p.tc = true;
  p.tc_fp8 = fp8 ? 1 : 0;
  p.tc_planes = fp8 ? 1 : planes;
  p.generic = true;
  p.npad = align_up(n, 4);
  p.kpad = align_up(k, 32);
  p.tc_kb = fp8 ? (n + 127) / 128 : (n + 63) / 64;   // 128-byte rows per K block
  p.tc_n16 = align_up(k, 16);
  p.tc_ncols = 32;
  while (p.tc_ncols < p.tc_n16) p.tc_ncols <<= 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BM_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = (int)std::max<long long>(1, std::min<long long>((s + 127) / 128, sms));
  if (cap > 0) grid = std::min(grid, cap);
  p.cap = cap;
  for (int iter = 0; iter < 16 && p.grid == 0; ++iter) {
    const int R = (int)((s + grid - 1) / grid);
    size_t smem = 0;
    int fb = 0, ns = 0;
    // widest staged block first, then a three-slot ring if it still fits
    for (int f : {64, 32, 16, 8, 4}) {
      for (int r : {3, 2}) {
        smem = chunk_tc_smem(p.npad, k, R, p.tc_n16, f, r, p.tc_planes);
        if (smem + 2048 <= kSmemLimit) { fb = f; ns = r; break; }   // + static smem
      }
      if (fb) break;
    }
    if (fb == 0) {   // too many rows per CTA: more CTAs, past the cap if need be
      if (grid >= sms) return BM_EUNSUPPORTED;
      grid = std::min(grid * 2, sms);
      continue;
    }
    const int maxg = chunk_tc_max_grid(smem);
    if (maxg <= 0) return BM_EUNSUPPORTED;
    if (grid > maxg) { grid = maxg; continue; }
    p.grid = grid;
    p.R = R;
    p.smem = smem;
    p.tc_fb = fb;
    p.tc_ns = ns;
    p.tc_tpc = (R + 127) / 128;
  }
  if (p.grid == 0) return BM_EUNSUPPORTED;
  // final assignment: the FP32 kernel when its tables fit, else tensor cores
  p.asmem = assign_smem(p.npad, k, p.kpad, true);
  p.agrid = p.asmem <= kSmemLimit ? assign_max_grid(true, 0, p.asmem) : 0;
  *out = p;
  return BM_OK;
}

static bm_status make_plan_simt(int n, int k, long long s, Plan* out, int cap);

// Kernel family for (n, k, s): the row-in-register path for n <= 32; for
// wider rows the tensor-core path when asked for (tc) or when the FP32
// tables do not fit in shared memory, else the tiled FP32 path.  planes: the
// tensor-core path's screening arithmetic (1: BF16, 2: split BF16); fp8:
// E4M3 screening instead.
// cap > 0 limits the CTAs of a chunk launch (the job then leaves the other
// SMs to concurrent jobs); it gives way where shared memory needs more CTAs.
static bm_status make_plan(int n, int k, long long s, Plan* out, bool tc = false, int cap = 0,
                           int planes = 2, bool fp8 = false) {
  if (n > kNpMax && tc) return make_plan_tc(n, k, s, out, cap, planes, fp8);
  const bm_status st = make_plan_simt(n, k, s, out, cap);
  if (st == BM_EUNSUPPORTED && n > kNpMax) return make_plan_tc(n, k, s, out, cap, planes, fp8);
  return st;
}

static bm_status make_plan_simt(int n, int k, long long s, Plan* out, int cap) {
  Plan p;
  if (k > kMaxK) return BM_EUNSUPPORTED;
  if (n <= kNpMax) {
    p.generic = false;
    p.np = np_width(n);
    p.npad = p.np;
    p.kpad = 0;
  } else {
    p.generic = true;
    p.np = 0;
    p.npad = align_up(n, 4);
    p.kpad = align_up(k, 32);
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BM_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // Grid: at most one CTA per SM, so that every SM carries the same share of
  // the sample, and at least 64 (row-in-register path) or 256 (tiled path)
  // rows per CTA so that small samples do not pay for idle CTAs in every
  // grid barrier.
  const int rows_target = p.generic ? 256 : 64;
  int grid = (int)std::min<long long>((s + rows_target - 1) / rows_target, (long long)sms);
  if (cap > 0) grid = std::min(grid, cap);
  grid = std::max(grid, 1);
  p.cap = cap;
  for (int iter = 0; iter < 8; ++iter) {
    const int R = (int)((s + grid - 1) / grid);
    const ChunkSmem L = chunk_smem(p.npad, k, p.kpad, R, p.generic);
    if ((size_t)L.total > kSmemLimit) {
      if (grid >= sms * 8) return BM_EUNSUPPORTED;
      grid = std::min(grid * 2, sms * 8);
      continue;
    }
    const int maxg = chunk_max_grid(p.generic, p.np, L.total);
    if (maxg <= 0) return BM_EUNSUPPORTED;
    if (grid > maxg) { grid = maxg; continue; }
    p.grid = grid;
    p.R = R;
    p.smem = L.total;
    break;
  }
  if (p.grid == 0) return BM_EUNSUPPORTED;
  p.asmem = assign_smem(p.npad, k, p.kpad, p.generic);
  if (p.asmem > kSmemLimit) return BM_EUNSUPPORTED;
  p.agrid = assign_max_grid(p.generic, p.np, p.asmem);
  if (p.agrid <= 0) return BM_EUNSUPPORTED;
  *out = p;
  return BM_OK;
}

// ------------------------------------------------------------ workspace
struct Workspace {
  int32_t* idx = nullptr;       // sample plan: [plan_cap][s] sorted rows
  uint32_t* bitmap = nullptr;   // [plan_cap][draw_bitmap_words(m)], zero between draws
  int plan_cap = 1;             // chunks drawn per sample-plan launch
  float* P = nullptr;
  float* C = nullptr;
  uint8_t* mask = nullptr;
  float* Cinc = nullptr;
  uint8_t* mask_inc = nullptr;
  double* f_opt = nullptr;
  float* part_sum = nullptr;
  int32_t* part_cnt = nullptr;
  double* part_f = nullptr;
  int32_t* blk_cnt = nullptr;
  Ctl* ctl = nullptr;
  Stats* stats = nullptr;
  unsigned long long* kx = nullptr;   // K-means++ exchange tags (ChunkArgs::kx)
  size_t kx_words = 0;
  double* apart = nullptr;   // assign per-CTA partials
  int apart_cap = 0;
  double* asse = nullptr;    // assign result
  unsigned long long* rescored = nullptr;  // tensor-core assign: rescored rows
  unsigned char* Cb = nullptr;  // tensor-core chunk kernel: centroid BF16 planes,
  float* sqs = nullptr;         // squared norms of 8-feature slices,
  unsigned char* Pb = nullptr;  // own-row BF16 planes
  std::vector<void*> owned;
  // allocation source: cudaMalloc, or a stream-ordered memory pool (serving:
  // no device-wide synchronisation per job, memory reused across jobs)
  cudaMemPool_t pool = nullptr;
  cudaStream_t pool_stream = nullptr;
  bool dry = false;     // only add up the bytes (footprint estimate)
  size_t bytes = 0;

  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    const size_t b = std::max<size_t>(count * sizeof(T), 16);
    bytes += (b + 511) / 512 * 512;
    if (dry) { *p = nullptr; return cudaSuccess; }
    void* v = nullptr;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&v, b, pool, pool_stream)
                               : cudaMalloc(&v, b);
    if (e != cudaSuccess) return e;
    owned.push_back(v);
    *p = static_cast<T*>(v);
    return cudaSuccess;
  }
  void release() {
    for (void* v : owned) {
      if (pool) cudaFreeAsync(v, pool_stream);
      else cudaFree(v);
    }
    owned.clear();
  }
};

// Chunks per sample-plan launch: up to 64, within 256 MB of plan memory.
static int plan_capacity(long long m, long long s) {
  const long long per = (long long)draw_bitmap_words(m) * 4 + s * 4;
  long long cap = (256LL << 20) / std::max<long long>(per, 1);
  return (int)std::max<long long>(1, std::min<long long>(64, cap));
}

static bm_status ws_create(Workspace* w, long long m, int k, long long s,
                           const Plan& p, cudaStream_t st, int plan_cap = 1,
                           long long assign_rows = 0) {
  const size_t words = draw_bitmap_words(m);
  const int G = p.grid;
  w->plan_cap = plan_cap;
  cudaError_t e = cudaSuccess;
#define BM_TRY(x) do { e = (x); if (e != cudaSuccess) { w->release(); return BM_ENOMEM; } } while (0)
  BM_TRY(w->alloc(&w->idx, (size_t)s * plan_cap));
  BM_TRY(w->alloc(&w->bitmap, words * plan_cap));
  BM_TRY(w->alloc(&w->P, (size_t)s * p.npad));
  BM_TRY(w->alloc(&w->C, (size_t)k * p.npad));
  BM_TRY(w->alloc(&w->mask, (size_t)k));
  BM_TRY(w->alloc(&w->Cinc, (size_t)k * p.npad));
  BM_TRY(w->alloc(&w->mask_inc, (size_t)k));
  BM_TRY(w->alloc(&w->f_opt, 1));
  BM_TRY(w->alloc(&w->part_sum, (size_t)k * p.npad * G));
  BM_TRY(w->alloc(&w->part_cnt, (size_t)k * G));
  BM_TRY(w->alloc(&w->part_f, (size_t)(kMaxTrials + 2) * G));
  BM_TRY(w->alloc(&w->blk_cnt, (size_t)G));
  BM_TRY(w->alloc(&w->ctl, 1));
  BM_TRY(w->alloc(&w->stats, 1));
  w->kx_words = 1 + 2 * (size_t)G + kMaxTrials;
  BM_TRY(w->alloc(&w->kx, w->kx_words));
  // assignment partials: per CTA (FP32 kernels) or per 128-row tile (tensor cores)
  w->apart_cap = (int)std::max<long long>(std::max(p.agrid, 4096), (assign_rows + 127) / 128);
  BM_TRY(w->alloc(&w->apart, (size_t)w->apart_cap));
  BM_TRY(w->alloc(&w->asse, 1));
  BM_TRY(w->alloc(&w->rescored, 1));
  const size_t cb_bytes = p.tc ? (size_t)p.tc_kb * 2 * p.tc_n16 * 128 : 16;
  if (p.tc) {
    BM_TRY(w->alloc(&w->Cb, cb_bytes));
    BM_TRY(w->alloc(&w->sqs, (size_t)k * ((p.npad + 7) / 8)));
    BM_TRY(w->alloc(&w->Pb, (size_t)p.grid * p.tc_tpc * p.tc_kb * p.tc_planes * 16384));
  }
#undef BM_TRY
  if (w->dry) return BM_OK;
  if (p.tc) cudaMemsetAsync(w->Cb, 0, cb_bytes, st);
  cudaMemsetAsync(w->bitmap, 0, words * 4 * plan_cap, st);
  cudaMemsetAsync(w->C, 0, (size_t)k * p.npad * 4, st);
  cudaMemsetAsync(w->Cinc, 0, (size_t)k * p.npad * 4, st);
  cudaMemsetAsync(w->mask, 0, k, st);
  cudaMemsetAsync(w->mask_inc, 0, k, st);
  cudaMemsetAsync(w->ctl, 0, sizeof(Ctl), st);
  cudaMemsetAsync(w->stats, 0, sizeof(Stats), st);
  cudaMemsetAsync(w->kx, 0, w->kx_words * 8, st);
  cudaMemsetAsync(w->part_f, 0, (size_t)(kMaxTrials + 2) * G * 8, st);
  const double inf = std::numeric_limits<double>::infinity();
  cudaMemcpyAsync(w->f_opt, &inf, sizeof(double), cudaMemcpyHostToDevice, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) { w->release(); return BM_ECUDA; }
  return BM_OK;
}

static ChunkArgs chunk_args(const Workspace& w, const Plan& p, const float* X,
                            long long m, int n, int k, long long s) {
  ChunkArgs a{};
  a.X = X; a.m = m; a.n = n; a.npad = p.npad; a.k = k; a.s = (int)s;
  a.rows_per_cta = p.R; a.kpad = p.kpad;
  a.max_iter = 300; a.tol = 1e-4; a.trials = 3;
  a.idx = w.idx; a.P = w.P; a.C = w.C; a.mask = w.mask;
  a.Cinc = w.Cinc; a.mask_inc = w.mask_inc; a.f_opt = w.f_opt;
  a.part_sum = w.part_sum; a.part_cnt = w.part_cnt; a.part_f = w.part_f;
  a.blk_cnt = w.blk_cnt; a.ctl = w.ctl; a.stats = w.stats; a.kx = w.kx;
  a.tc_kb = p.tc_kb; a.tc_n16 = p.tc_n16; a.tc_ncols = p.tc_ncols; a.tc_fb = p.tc_fb;
  a.tc_tpc = p.tc_tpc; a.tc_ns = p.tc_ns; a.tc_planes = p.tc_planes; a.tc_fp8 = p.tc_fp8;
  a.Cb = w.Cb; a.sqs = w.sqs; a.Pb = w.Pb;
  return a;
}

// One chunk-kernel launch of the plan's family.
static cudaError_t launch_plan(const ChunkArgs& a, const Plan& p, cudaStream_t st) {
  if (p.tc) return launch_chunk_tc(a, p.grid, p.smem, st);
  return launch_chunk(a, p.grid, p.generic, p.np, p.smem, st);
}

static bool shape_ok(long long m, int n, int k, long long s) {
  const long long lim = 2147483647LL;
  return m >= 1 && n >= 1 && k >= 1 && s >= 1 && s <= m && k <= s && m <= lim &&
         s <= lim;
}

// Reads the status word; on error clears the control block so that the
// workspace can be used again.
// K-means++ exchange reads that found their value not yet published (each
// waited for it), summed over every launch checked since the library loaded.
static std::atomic<unsigned long long> g_late_reads{0};

static bm_status check_status(Workspace& w, cudaStream_t st, long long m) {
  (void)m;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return BM_ECUDA;
  Ctl h{};
  e = cudaMemcpy(&h, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return BM_ECUDA;
  if (h.late != 0) {
    g_late_reads += h.late;
    const uint32_t zero = 0;
    if (cudaMemcpy(&w.ctl->late, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
      return BM_ECUDA;
  }
  if (h.status != 0) {
    // an aborted launch may leave barrier counters and exchange tags behind
    cudaMemset(w.ctl, 0, sizeof(Ctl));
    if (w.kx) cudaMemset(w.kx, 0, w.kx_words * 8);
    cudaDeviceSynchronize();
    return (bm_status)h.status;
  }
  return BM_OK;
}

}  // namespace bm

using namespace bm;

// ====================================================================== ctx
// A recorded bm_fit_chunk launch sequence and the launch state it starts
// from and ends in.
struct FitGraph {
  long long t, chunks, parity, plan_t0, plan_n;   // state before
  long long end_plan_t0, end_plan_n;              // sample-plan window after
  cudaGraphExec_t exec;
  long long stamp;                                // last use (eviction order)
};

struct bm_ctx {
  bm_config cfg;
  const float* X;
  // bm_fit_host while its copy of X is in flight: the device-accessible host
  // rows, the count of landed copy pieces and the pieces' block size
  // (2^x_shift rows); null otherwise
  const float* Xh = nullptr;
  const uint32_t* x_ready = nullptr;
  int x_shift = 0;
  cudaStream_t stream;
  Plan plan;
  Workspace ws;
  long long t = 0;          // next chunk index
  long long launches = 0;   // selects the barrier counter
  long long plan_t0 = -1;   // first chunk held by the sample plan (-1: none)
  long long plan_n = 0;     // chunks held by the sample plan
  long long nd_assign = 0;  // distance evaluations of bm_assign calls
  unsigned long long rescored = 0;  // rows rescored by the last tensor-core bm_assign
  // full-data Lloyd polish: labels and per-CTA partials, allocated on first use
  int32_t* pol_labels = nullptr;
  float* pol_sum = nullptr;
  int32_t* pol_cnt = nullptr;
  int pol_grid = 0;
  std::vector<FitGraph> graphs;     // recorded fits, at most kMaxGraphs
  long long graph_clock = 0;
  bool graphs_ok = true;            // cleared if recording ever fails
  std::mutex mu;
};

static constexpr size_t kMaxGraphs = 4;

namespace bm {

static bm_status check_config(const bm_config* cfg) {
  if (!shape_ok(cfg->m, cfg->n, cfg->k, cfg->s)) return BM_EINVAL;
  if (cfg->kpp_trials < 1 || cfg->kpp_trials > kMaxTrials || cfg->max_iter < 0 ||
      !(cfg->tol >= 0.0))
    return BM_EINVAL;
  if (cfg->precision != BM_FP32 && cfg->precision != BM_BF16_RESCORE &&
      cfg->precision != BM_BF16X3_RESCORE && cfg->precision != BM_FP8_RESCORE)
    return BM_EUNSUPPORTED;
  if (cfg->init != BM_INIT_KMEANSPP && cfg->init != BM_INIT_FORGY) return BM_EINVAL;
  if (cfg->empty != BM_EMPTY_DEGENERATE && cfg->empty != BM_EMPTY_KEEP) return BM_EINVAL;
  return BM_OK;
}

static bool wants_tc(const bm_config* cfg) {
  return cfg->precision == BM_BF16_RESCORE || cfg->precision == BM_BF16X3_RESCORE ||
         cfg->precision == BM_FP8_RESCORE;
}

// Screening arithmetic of the tensor-core chunk kernel for a precision
// form: BF16 products (one plane), E4M3 products, or split BF16 (two planes)
// for the others.
static int chunk_planes(int precision) {
  return precision == BM_BF16_RESCORE || precision == BM_FP8_RESCORE ? 1 : 2;
}
static bool chunk_fp8(int precision) { return precision == BM_FP8_RESCORE; }

// Screening arithmetic of the tensor-core final assignment for a precision
// form.
static int assign_terms(int precision) {
  return precision == BM_BF16_RESCORE ? 1 : precision == BM_FP8_RESCORE ? kTermsFp8 : 3;
}

bm_status ctx_create(const bm_config* cfg, const float* X_dev, cudaStream_t stream,
                     cudaMemPool_t pool, bm_ctx** out, int plan_cap) {
  if (!cfg || !out || (!X_dev && plan_cap >= 0)) return BM_EINVAL;   // plan_cap < 0: no X
  *out = nullptr;
  bm_status st = check_config(cfg);
  if (st != BM_OK) return st;
  bm_ctx* c = new (std::nothrow) bm_ctx();
  if (!c) return BM_ENOMEM;
  c->cfg = *cfg;
  c->X = X_dev;
  c->stream = stream;
  st = make_plan(cfg->n, cfg->k, cfg->s, &c->plan, wants_tc(cfg), cfg->max_ctas,
                 chunk_planes(cfg->precision), chunk_fp8(cfg->precision));
  if (st != BM_OK) { delete c; return st; }
  c->ws.pool = pool;
  c->ws.pool_stream = stream;
  st = ws_create(&c->ws, cfg->m, cfg->k, cfg->s, c->plan, c->stream,
                 plan_cap > 0 ? plan_cap : plan_cap < 0 ? 1 : plan_capacity(cfg->m, cfg->s),
                 cfg->m);
  if (st != BM_OK) { delete c; return st; }
  *out = c;
  return BM_OK;
}

bm_status ctx_footprint(const bm_config* cfg, size_t* bytes) {
  if (!cfg || !bytes) return BM_EINVAL;
  bm_status st = check_config(cfg);
  if (st != BM_OK) return st;
  Plan p;
  st = make_plan(cfg->n, cfg->k, cfg->s, &p, wants_tc(cfg), cfg->max_ctas,
                 chunk_planes(cfg->precision), chunk_fp8(cfg->precision));
  if (st != BM_OK) return st;
  Workspace w;
  w.dry = true;
  st = ws_create(&w, cfg->m, cfg->k, cfg->s, p, nullptr, plan_capacity(cfg->m, cfg->s), cfg->m);
  if (st != BM_OK) return st;
  *bytes = w.bytes;
  return BM_OK;
}

}  // namespace bm

extern "C" {

void bm_config_default(bm_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->max_iter = 300;
  cfg->tol = 1e-4;
  cfg->kpp_trials = 3;
  cfg->seed = 0;
  cfg->precision = BM_FP32;
  cfg->time_budget_s = 0.0;
  cfg->graphs = 1;
  cfg->trace = 0;
  cfg->max_ctas = 0;
  cfg->init = BM_INIT_KMEANSPP;
  cfg->empty = BM_EMPTY_DEGENERATE;
}

uint64_t bm_sync_late_reads(void) { return g_late_reads.load(); }

const char* bm_status_string(int32_t s) {
  switch (s) {
    case BM_OK: return "ok";
    case BM_EINVAL: return "invalid argument";
    case BM_ENOMEM: return "out of device memory";
    case BM_ECUDA: return "CUDA error";
    case BM_ETIMEOUT: return "device wait timed out";
    case BM_EBUSY: return "busy";
    case BM_ECANCELLED: return "cancelled";
    case BM_EUNSUPPORTED: return "unsupported shape";
    case BM_EGUARD: return "device index guard tripped (debug build)";
    default: return "unknown status";
  }
}

bm_status bm_create(const bm_config* cfg, const float* X_dev, void* stream,
                    bm_ctx** out) {
  return bm::ctx_create(cfg, X_dev, static_cast<cudaStream_t>(stream), nullptr, out);
}

bm_status bm_destroy(bm_ctx* c) {
  if (!c) return BM_OK;
  cudaStreamSynchronize(c->stream);
  for (FitGraph& g : c->graphs) cudaGraphExecDestroy(g.exec);
  if (c->pol_labels) cudaFree(c->pol_labels);
  if (c->pol_sum) cudaFree(c->pol_sum);
  if (c->pol_cnt) cudaFree(c->pol_cnt);
  c->ws.release();
  delete c;
  return BM_OK;
}

bm_status bm_reset(bm_ctx* c) {
  if (!c) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const int k = c->cfg.k;
  cudaStream_t st = c->stream;
  cudaMemsetAsync(c->ws.Cinc, 0, (size_t)k * c->plan.npad * 4, st);
  cudaMemsetAsync(c->ws.mask_inc, 0, k, st);
  cudaMemsetAsync(c->ws.ctl, 0, sizeof(Ctl), st);
  cudaMemsetAsync(c->ws.stats, 0, sizeof(Stats), st);
  const size_t words = draw_bitmap_words(c->cfg.m);
  cudaMemsetAsync(c->ws.bitmap, 0, words * 4 * c->ws.plan_cap, st);
  c->plan_t0 = -1;
  static const double inf = std::numeric_limits<double>::infinity();
  cudaMemcpyAsync(c->ws.f_opt, &inf, sizeof(double), cudaMemcpyHostToDevice, st);
  c->t = 0;
  c->launches = 0;
  c->nd_assign = 0;
  return cudaStreamSynchronize(st) == cudaSuccess ? BM_OK : BM_ECUDA;
}

// Queues the launches of `chunks` chunks from c->t (sample-plan draws as
// the chunk index leaves the drawn window, one chunk launch per chunk) and
// advances the host-side launch state.  `left` < 0: as many as `chunks`.
static bm_status queue_chunks(bm_ctx* c, ChunkArgs a, long long chunks, long long left) {
  for (long long done = 0; done < chunks; ++done) {
    // the sample plan holds chunks [plan_t0, plan_t0 + plan_n)
    if (c->plan_t0 < 0 || c->t < c->plan_t0 || c->t >= c->plan_t0 + c->plan_n) {
      DrawArgs d{};
      d.m = c->cfg.m; d.s = (int)c->cfg.s; d.seed = c->cfg.seed; d.t0 = c->t;
      d.idx = c->ws.idx; d.bitmaps = c->ws.bitmap; d.status = &c->ws.ctl->status;
      int batch = c->ws.plan_cap;
      if (left >= 0) batch = (int)std::min<long long>(batch, left - done);
      if (launch_draw(d, batch, c->stream) != cudaSuccess) return BM_ECUDA;
      c->plan_t0 = c->t;
      c->plan_n = batch;
    }
    a.idx = c->ws.idx + (size_t)(c->t - c->plan_t0) * c->cfg.s;
    a.t = c->t;
    a.bar_sel = (int)(c->launches & 1);
    if (launch_plan(a, c->plan, c->stream) != cudaSuccess) return BM_ECUDA;
    ++c->launches;
    ++c->t;
  }
  return BM_OK;
}

// Replays (recording first if needed) the launch sequence of `chunks`
// chunks from the current state as one CUDA graph.  Returns false when
// recording is not possible; the state is then unchanged.
static bool fit_by_graph(bm_ctx* c, const ChunkArgs& a, long long chunks, bm_status* st) {
  const long long parity = c->launches & 1;
  FitGraph* hit = nullptr;
  for (FitGraph& g : c->graphs)
    if (g.t == c->t && g.chunks == chunks && g.parity == parity && g.plan_t0 == c->plan_t0 &&
        g.plan_n == c->plan_n)
      hit = &g;
  if (!hit) {
    const long long t0 = c->t, l0 = c->launches, p0 = c->plan_t0, n0 = c->plan_n;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const bm_status qs = queue_chunks(c, a, chunks, chunks);
    const cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    const bool ok = qs == BM_OK && ce == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    FitGraph g{t0, chunks, parity, p0, n0, c->plan_t0, c->plan_n, exec, 0};
    c->t = t0; c->launches = l0; c->plan_t0 = p0; c->plan_n = n0;   // nothing ran yet
    if (!ok) {
      cudaGetLastError();
      return false;
    }
    if (c->graphs.size() >= kMaxGraphs) {
      auto old = std::min_element(c->graphs.begin(), c->graphs.end(),
                                  [](const FitGraph& x, const FitGraph& y) { return x.stamp < y.stamp; });
      cudaGraphExecDestroy(old->exec);
      c->graphs.erase(old);
    }
    c->graphs.push_back(g);
    hit = &c->graphs.back();
  }
  hit->stamp = ++c->graph_clock;
  *st = cudaGraphLaunch(hit->exec, c->stream) == cudaSuccess ? BM_OK : BM_ECUDA;
  c->t += chunks;
  c->launches += chunks;
  c->plan_t0 = hit->end_plan_t0;
  c->plan_n = hit->end_plan_n;
  return true;
}

bm_status bm_fit_chunk(bm_ctx* c, int32_t chunks, bm_fit_report* out) {
  if (!c || chunks < 0 || !c->X) return BM_EINVAL;   // streaming contexts have no X
  if (chunks == 0 && !(c->cfg.time_budget_s > 0.0)) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const auto t0 = std::chrono::steady_clock::now();
  Stats before{};
  if (cudaMemcpyAsync(&before, c->ws.stats, sizeof(Stats), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return BM_ECUDA;
  ChunkArgs a = chunk_args(c->ws, c->plan, c->X, c->cfg.m, c->cfg.n, c->cfg.k, c->cfg.s);
  a.Xh = c->Xh;
  a.x_ready = c->x_ready;
  a.x_shift = c->x_shift;
  a.seed = c->cfg.seed;
  a.max_iter = c->cfg.max_iter;
  a.tol = c->cfg.tol;
  a.trials = c->cfg.kpp_trials;
  a.phases = kPhaseGather | kPhaseKpp | kPhaseLloyd | kPhaseKeep;
  a.trace = c->cfg.trace != 0;
  a.init = c->cfg.init;
  a.empty_keep = c->cfg.empty == BM_EMPTY_KEEP;
  bm_status st = BM_OK;
  if (chunks > 0) {
    // graph replay needs a capturable stream (not the legacy default stream)
    const bool graphed = c->cfg.graphs && c->graphs_ok && c->stream != nullptr &&
                         fit_by_graph(c, a, chunks, &st);
    if (!graphed) {
      if (c->cfg.graphs && c->stream != nullptr) c->graphs_ok = false;
      st = queue_chunks(c, a, chunks, chunks);
    }
  } else {
    // the paper's time budget (Sec. 5): chunks until the budget has elapsed.
    // One chunk stays queued ahead of the one the host waits for, so the GPU
    // never idles while the host reads the clock; the chunk queued when the
    // budget runs out still completes.
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess)
      st = BM_ECUDA;
    for (long long q = 0; st == BM_OK; ++q) {
      st = queue_chunks(c, a, 1, -1);
      if (st != BM_OK) break;
      if (cudaEventRecord(ev[q & 1], c->stream) != cudaSuccess) { st = BM_ECUDA; break; }
      if (q == 0) continue;   // two chunks in flight before the first wait
      if (cudaEventSynchronize(ev[(q - 1) & 1]) != cudaSuccess) { st = BM_ECUDA; break; }
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el >= c->cfg.time_budget_s) break;
    }
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  const bm_status st2 = check_status(c->ws, c->stream, c->cfg.m);
  if (st == BM_OK) st = st2;
  if (st != BM_OK) return st;
  if (out) {
    Stats after{};
    double f_opt = 0.0;
    cudaMemcpy(&after, c->ws.stats, sizeof(Stats), cudaMemcpyDeviceToHost);
    cudaMemcpy(&f_opt, c->ws.f_opt, sizeof(double), cudaMemcpyDeviceToHost);
    out->chunks = after.chunks - before.chunks;
    out->accepted = after.accepted - before.accepted;
    out->lloyd_iters = after.lloyd_iters - before.lloyd_iters;
    out->n_d = after.n_d + c->nd_assign;
    out->chunk_counter = c->t;
    out->f_opt = f_opt;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    out->host_gathers = after.host_gathers - before.host_gathers;
  }
  return BM_OK;
}

static bm_status assign_impl(const float* X, long long m, int n, int k,
                             const Plan& p, const float* C, int cstride,
                             const uint8_t* mask, int32_t* labels, float* dmin,
                             Workspace& w, cudaStream_t st, double* sse_out) {
  AssignArgs a{};
  a.X = X; a.m = m; a.n = n; a.npad = p.npad; a.k = k; a.kpad = p.kpad;
  a.C = C; a.cstride = cstride; a.mask = mask; a.labels = labels; a.dmin = dmin;
  a.part = w.apart; a.sse = w.asse; a.ticket = &w.ctl->assign_ticket;
  a.status = &w.ctl->status;
  const long long rows_per = p.generic ? 64 : 256;  // rows per CTA pass
  int grid = (int)std::max<long long>(1, std::min<long long>(p.agrid, (m + rows_per - 1) / rows_per));
  if (p.cap > 0) grid = std::min(grid, p.cap * std::max(1, p.agrid / std::max(1, sm_count())));
  if (launch_assign(a, grid, p.generic, p.np, p.asmem, st) != cudaSuccess) return BM_ECUDA;
  double sse = 0.0;
  if (cudaMemcpyAsync(&sse, w.asse, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return BM_ECUDA;
#ifdef BM_DEBUG_GUARDS
  const bm_status gs = check_status(w, st, m);   // an index guard that tripped
  if (gs != BM_OK) return gs;
#endif
  if (sse_out) *sse_out = sse;
  return BM_OK;
}

// Grid autotuner of the tensor-core assignment.  The best number of CTAs per
// SM depends on (n, MMA width, form): more CTAs overlap one tile's loads with another
// tile's MMA and epilogue, until shared memory, TMEM or the tail of the
// tile queue costs more.  The first call of a shape on a device times every
// candidate on the caller's own data and keeps the fastest; results do not
// depend on the grid (per-tile partial sums), so any candidate's output is
// the call's output.
}  // extern "C"

template <typename Launch>
static int tc_tuned_grid(int n, int k, int terms, int stages, int maxg, long long tiles,
                         Launch launch, cudaStream_t st) {
  static std::mutex mu;
  // (dev, n, MMA width, terms): k enters the kernel's cost through the MMA
  // width (k rounded up to 16), so shapes that share it share the choice
  static std::map<std::tuple<int, int, int, int>, int> best;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const auto key = std::make_tuple(dev, n, (k + 15) / 16, terms * 4 + stages);
  {
    std::lock_guard<std::mutex> g(mu);
    auto itr = best.find(key);
    if (itr != best.end()) return (int)std::min<long long>(itr->second, tiles);
  }
  const int per_max = std::max(1, maxg / sms);
  int pick = maxg;
  float pick_ms = 1e30f;
  if (tiles >= (long long)sms * 4) {   // enough work to tell candidates apart
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int per = 1; per <= per_max; ++per) {
      const int g = sms * per;
      cudaEventRecord(e0, st);
      if (launch(g) != cudaSuccess) break;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < pick_ms) { pick_ms = ms; pick = g; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> g(mu);
    best[key] = pick;
  }
  return (int)std::max<long long>(1, std::min<long long>(pick, tiles));
}

extern "C" {

// Tensor-core assignment (BF16 distances, exact FP32 rescoring).
static bm_status assign_tc_impl(const float* X, long long m, int n, int k,
                                const float* C, int cstride, const uint8_t* mask,
                                int32_t* labels, float* dmin, Workspace& w,
                                cudaStream_t st, double* sse_out,
                                unsigned long long* rescored_out, int terms, int cap = 0) {
  if (k > kMaxK) return BM_EUNSUPPORTED;
  int stages, kb, npad16, ncols, cf;
  // room for the kernel's static shared memory and the per-CTA reservation
  const size_t limit = kSmemLimit - 2048;
  {
    // rows of at most 128 features: the streaming kernel, one persistent CTA
    // per SM (TMA column boxes, rows held in registers)
    TcsPlan tp{};
    const size_t ssmem = assign_tcs_plan(n, k, terms, limit, &tp);
    const long long tiles = (m + 127) / 128;
    if (terms != kTermsFp8 && ssmem > 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
        tiles <= w.apart_cap && m < (1LL << 31)) {
      int sms = 0, dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      int grid = (int)std::min<long long>(tiles, sms);
      if (cap > 0) grid = std::min(grid, cap);
      if (cudaMemsetAsync(w.rescored, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return BM_ECUDA;
      const cudaError_t e = launch_assign_tcs(
          X, m, n, C, cstride, mask, k, labels, dmin, reinterpret_cast<float2*>(w.apart), w.asse,
          &w.ctl->assign_ticket, w.rescored, &w.ctl->status, terms, tp, ssmem, grid, st);
      if (e == cudaSuccess) {
        double sse = 0.0;
        unsigned long long resc = 0;
        if (cudaMemcpyAsync(&sse, w.asse, sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(&resc, w.rescored, sizeof(resc), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess)
          return BM_ECUDA;
        const bm_status rc = check_status(w, st, 0);
        if (rc != BM_OK) return rc;
        if (sse_out) *sse_out = sse;
        if (rescored_out) *rescored_out = resc;
        return BM_OK;
      }
      if (e != cudaErrorNotSupported && e != cudaErrorInvalidValue &&
          e != cudaErrorLaunchOutOfResources)
        return BM_ECUDA;
      cudaGetLastError();   // no tensor-map encoder: the tiled kernel below
    }
  }
  // bulk copies of row tiles need a 16-byte aligned X
  const bool bulk_ok = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  size_t smem = assign_tc_smem(n, k, terms, &stages, &kb, &npad16, &ncols, &cf, bulk_ok, limit);
  if (smem > limit && terms == 3) {   // the split form does not fit: one term
    terms = 1;
    smem = assign_tc_smem(n, k, terms, &stages, &kb, &npad16, &ncols, &cf, bulk_ok, limit);
  }
  if (smem > limit) return BM_EUNSUPPORTED;
  int maxg = assign_tc_max_grid(smem, terms);
  if (maxg <= 0) return BM_EUNSUPPORTED;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  maxg = std::min(maxg, sms * std::max(1, 512 / ncols));   // TMEM columns per SM
  const long long tiles = (m + 127) / 128;
  if (tiles > w.apart_cap) return BM_EUNSUPPORTED;
  const int grid = tc_tuned_grid(n, k, terms, stages, maxg, tiles, [&](int g) {
    AssignTcArgs t{};
    t.X = X; t.m = m; t.n = n; t.C = C; t.cstride = cstride; t.mask = mask; t.k = k;
    t.labels = labels; t.dmin = dmin; t.part = reinterpret_cast<float2*>(w.apart);
    t.sse = w.asse; t.ticket = &w.ctl->assign_ticket; t.rescored = w.rescored;
    t.status = &w.ctl->status; t.kb = kb; t.npad16 = npad16; t.ncols = ncols;
    t.stages = stages; t.use_bulk = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    t.terms = terms; t.cf = cf;
    return launch_assign_tc(t, g, smem, st);
  }, st);
  const int launch_grid = cap > 0 ? std::min(grid, cap * std::max(1, maxg / sms)) : grid;
  AssignTcArgs a{};
  a.X = X; a.m = m; a.n = n; a.C = C; a.cstride = cstride; a.mask = mask; a.k = k;
  a.labels = labels; a.dmin = dmin; a.part = reinterpret_cast<float2*>(w.apart);
  a.sse = w.asse;
  a.ticket = &w.ctl->assign_ticket; a.rescored = w.rescored; a.status = &w.ctl->status;
  a.kb = kb; a.npad16 = npad16; a.ncols = ncols; a.stages = stages;
  a.use_bulk = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  a.terms = terms;
  a.cf = cf;
  if (cudaMemsetAsync(w.rescored, 0, sizeof(unsigned long long), st) != cudaSuccess) return BM_ECUDA;
  if (launch_assign_tc(a, launch_grid, smem, st) != cudaSuccess) return BM_ECUDA;
  double sse = 0.0;
  unsigned long long resc = 0;
  if (cudaMemcpyAsync(&sse, w.asse, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&resc, w.rescored, sizeof(resc), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BM_ECUDA;
  const bm_status rc = check_status(w, st, 0);
  if (rc != BM_OK) return rc;
  if (sse_out) *sse_out = sse;
  if (rescored_out) *rescored_out = resc;
  return BM_OK;
}

static int count_live_host(const uint8_t* mask_dev, int k, cudaStream_t st) {
  std::vector<uint8_t> h(k);
  if (cudaMemcpyAsync(h.data(), mask_dev, k, cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  int n = 0;
  for (uint8_t v : h) n += v != 0;
  return n;
}

bm_status bm_assign(bm_ctx* c, int32_t* labels_dev, double* sse_out) {
  if (!c || !c->X) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const int live = count_live_host(c->ws.mask_inc, c->cfg.k, c->stream);
  if (live < 0) return BM_ECUDA;
  if (live == 0) return BM_EINVAL;   // no incumbent yet
  bm_status st;
  // FP32 results from the tensor cores too when the FP32 kernel's tables do
  // not fit (the rescoring makes the labels and distances those of FP32)
  if (wants_tc(&c->cfg) ||
      c->plan.agrid == 0)
    st = assign_tc_impl(c->X, c->cfg.m, c->cfg.n, c->cfg.k, c->ws.Cinc, c->plan.npad,
                        c->ws.mask_inc, labels_dev, nullptr, c->ws, c->stream, sse_out,
                        &c->rescored, assign_terms(c->cfg.precision),
                        c->plan.cap);
  else
    st = assign_impl(c->X, c->cfg.m, c->cfg.n, c->cfg.k, c->plan, c->ws.Cinc,
                     c->plan.npad, c->ws.mask_inc, labels_dev, nullptr, c->ws,
                     c->stream, sse_out);
  if (st == BM_OK) c->nd_assign += c->cfg.m * (long long)live;
  return st;
}

// The paper's parallel modes 2 and 3 (Sec. 3.5) on one GPU: W worker
// contexts on their own streams, each capped at SMs / W CTAs so the workers
// run side by side; worker w processes chunk t0 + r W + w in round r (one
// sample each; a worker's sample plan holds one chunk).  Competitive: every
// worker keeps its own incumbent (starting from the context's) and the best
// incumbent -- lowest f_opt, lowest worker on ties -- becomes the context's
// at the end.  Collective: every round starts all workers from the context's
// incumbent and the best of their results replaces it when strictly better.
bm_status bm_fit_workers(bm_ctx* c, int32_t workers, int32_t rounds, int32_t mode,
                         bm_fit_report* out) {
  if (!c || !c->X || workers < 1 || rounds < 0 || (mode != BM_WORKERS_COMPETITIVE &&
                                          mode != BM_WORKERS_COLLECTIVE))
    return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const auto t_begin = std::chrono::steady_clock::now();
  const int k = c->cfg.k, npad = c->plan.npad;
  const size_t cbytes = (size_t)k * npad * 4;
  bm_config wcfg = c->cfg;
  wcfg.graphs = 0;
  wcfg.trace = 0;
  if (wcfg.max_ctas <= 0) wcfg.max_ctas = (sm_count() + workers - 1) / workers;
  std::vector<bm_ctx*> w(workers, nullptr);
  std::vector<cudaStream_t> ws(workers, nullptr);
  bm_status rc = BM_OK;
  auto cleanup = [&]() {
    for (int i = 0; i < workers; ++i) {
      if (w[i]) bm_destroy(w[i]);
      if (ws[i]) cudaStreamDestroy(ws[i]);
    }
  };
  // copies of (C_inc, mask_inc, f_opt) between contexts, on `st`
  auto copy_inc = [&](bm_ctx* dst, const bm_ctx* src, cudaStream_t st) {
    return cudaMemcpyAsync(dst->ws.Cinc, src->ws.Cinc, cbytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(dst->ws.mask_inc, src->ws.mask_inc, k, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(dst->ws.f_opt, src->ws.f_opt, 8, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
  };
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return BM_ECUDA;
  for (int i = 0; i < workers && rc == BM_OK; ++i) {
    if (cudaStreamCreateWithFlags(&ws[i], cudaStreamNonBlocking) != cudaSuccess) rc = BM_ECUDA;
    else rc = ctx_create(&wcfg, c->X, ws[i], nullptr, &w[i], 1);
    if (rc == BM_OK && !copy_inc(w[i], c, ws[i])) rc = BM_ECUDA;
  }
  if (rc != BM_OK) { cleanup(); return rc; }
  const long long t0 = c->t;
  std::vector<double> fo(workers);
  for (int r = 0; r < rounds && rc == BM_OK; ++r) {
    for (int i = 0; i < workers && rc == BM_OK; ++i) {
      bm_ctx* x = w[i];
      if (mode == BM_WORKERS_COLLECTIVE && r > 0 && !copy_inc(x, c, x->stream)) rc = BM_ECUDA;
      ChunkArgs a = chunk_args(x->ws, x->plan, x->X, x->cfg.m, x->cfg.n, k, x->cfg.s);
      a.seed = x->cfg.seed; a.max_iter = x->cfg.max_iter; a.tol = x->cfg.tol;
      a.trials = x->cfg.kpp_trials;
      a.init = x->cfg.init;
      a.empty_keep = x->cfg.empty == BM_EMPTY_KEEP;
      a.phases = kPhaseGather | kPhaseKpp | kPhaseLloyd | kPhaseKeep;
      x->t = t0 + (long long)r * workers + i;
      if (rc == BM_OK) rc = queue_chunks(x, a, 1, 1);
    }
    for (int i = 0; i < workers; ++i) {
      const bm_status s2 = check_status(w[i]->ws, w[i]->stream, 0);
      if (rc == BM_OK) rc = s2;
    }
    if (rc != BM_OK || mode != BM_WORKERS_COLLECTIVE) continue;
    // the round's best result replaces the shared incumbent when strictly better
    double f_best = 0.0;
    if (cudaMemcpy(&f_best, c->ws.f_opt, 8, cudaMemcpyDeviceToHost) != cudaSuccess) { rc = BM_ECUDA; break; }
    int best = -1;
    for (int i = 0; i < workers; ++i) {
      if (cudaMemcpy(&fo[i], w[i]->ws.f_opt, 8, cudaMemcpyDeviceToHost) != cudaSuccess) { rc = BM_ECUDA; break; }
      if (fo[i] < f_best && (best < 0 || fo[i] < fo[best])) best = i;
    }
    if (rc == BM_OK && best >= 0 &&
        (!copy_inc(c, w[best], c->stream) || cudaStreamSynchronize(c->stream) != cudaSuccess))
      rc = BM_ECUDA;
  }
  if (rc == BM_OK && mode == BM_WORKERS_COMPETITIVE) {
    int best = -1;
    for (int i = 0; i < workers && rc == BM_OK; ++i) {
      if (cudaMemcpy(&fo[i], w[i]->ws.f_opt, 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = BM_ECUDA;
      else if (best < 0 || fo[i] < fo[best]) best = i;
    }
    double f_c = 0.0;
    if (rc == BM_OK && cudaMemcpy(&f_c, c->ws.f_opt, 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = BM_ECUDA;
    if (rc == BM_OK && best >= 0 && fo[best] < f_c &&
        (!copy_inc(c, w[best], c->stream) || cudaStreamSynchronize(c->stream) != cudaSuccess))
      rc = BM_ECUDA;
  }
  Stats tot{};
  for (int i = 0; i < workers && rc == BM_OK; ++i) {
    Stats h{};
    if (cudaMemcpy(&h, w[i]->ws.stats, sizeof(Stats), cudaMemcpyDeviceToHost) != cudaSuccess) { rc = BM_ECUDA; break; }
    tot.chunks += h.chunks;
    tot.accepted += h.accepted;
    tot.lloyd_iters += h.lloyd_iters;
    tot.n_d += h.n_d;
  }
  cleanup();
  if (rc != BM_OK) return rc;
  c->t = t0 + (long long)rounds * workers;
  c->nd_assign += tot.n_d;   // the workers' distance evaluations count for this context
  if (out) {
    double f_opt = 0.0;
    cudaMemcpy(&f_opt, c->ws.f_opt, 8, cudaMemcpyDeviceToHost);
    Stats mine{};
    cudaMemcpy(&mine, c->ws.stats, sizeof(Stats), cudaMemcpyDeviceToHost);
    out->chunks = tot.chunks;
    out->accepted = tot.accepted;
    out->lloyd_iters = tot.lloyd_iters;
    out->n_d = mine.n_d + c->nd_assign;
    out->chunk_counter = c->t;
    out->f_opt = f_opt;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_begin).count();
  }
  return BM_OK;
}

// Streaming (no resident X): each pushed portion of rows is one chunk's
// sample.  The context is a normal one sized for portions of up to cfg.s
// rows, whose sample buffer P receives the portion instead of a gather.
bm_status bm_stream_create(const bm_config* cfg, void* stream, bm_ctx** out) {
  if (!cfg || !out) return BM_EINVAL;
  bm_config c2 = *cfg;
  c2.m = cfg->s;   // sizes the per-chunk state only
  c2.graphs = 0;
  bm_status st = ctx_create(&c2, nullptr, static_cast<cudaStream_t>(stream), nullptr, out, -1);
  if (st != BM_OK) return st;
  bm_ctx* c = *out;
  // P's padding columns stay zero: portions fill only the first n columns
  if (cudaMemsetAsync(c->ws.P, 0, (size_t)c->cfg.s * c->plan.npad * 4, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    bm_destroy(c);
    *out = nullptr;
    return BM_ECUDA;
  }
  return BM_OK;
}

bm_status bm_stream_push(bm_ctx* c, const float* P_dev, int64_t rows, bm_fit_report* out) {
  if (!c || c->X || !P_dev || rows < c->cfg.k || rows > c->cfg.s) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const auto t0 = std::chrono::steady_clock::now();
  const int n = c->cfg.n, npad = c->plan.npad;
  cudaStream_t st = c->stream;
  Stats before{};
  if (cudaMemcpyAsync(&before, c->ws.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpy2DAsync(c->ws.P, npad * 4, P_dev, n * 4, n * 4, rows, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return BM_ECUDA;
  ChunkArgs a = chunk_args(c->ws, c->plan, nullptr, rows, n, c->cfg.k, rows);
  a.rows_per_cta = c->plan.R;   // the plan's shape, fewer rows
  a.seed = c->cfg.seed; a.max_iter = c->cfg.max_iter; a.tol = c->cfg.tol;
  a.trials = c->cfg.kpp_trials; a.init = c->cfg.init; a.trace = c->cfg.trace != 0;
  a.empty_keep = c->cfg.empty == BM_EMPTY_KEEP;
  a.phases = kPhaseKpp | kPhaseLloyd | kPhaseKeep;
  a.t = c->t;
  a.bar_sel = (int)(c->launches & 1);
  bm_status rc = launch_plan(a, c->plan, st) == cudaSuccess ? BM_OK : BM_ECUDA;
  if (rc == BM_OK) {
    ++c->launches;
    ++c->t;
  }
  const bm_status s2 = check_status(c->ws, st, rows);
  if (rc == BM_OK) rc = s2;
  if (rc != BM_OK) return rc;
  if (out) {
    Stats after{};
    double f_opt = 0.0;
    cudaMemcpy(&after, c->ws.stats, sizeof(Stats), cudaMemcpyDeviceToHost);
    cudaMemcpy(&f_opt, c->ws.f_opt, sizeof(double), cudaMemcpyDeviceToHost);
    out->chunks = after.chunks - before.chunks;
    out->accepted = after.accepted - before.accepted;
    out->lloyd_iters = after.lloyd_iters - before.lloyd_iters;
    out->n_d = after.n_d;
    out->chunk_counter = c->t;
    out->f_opt = f_opt;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return BM_OK;
}

bm_status bm_polish(bm_ctx* c, int32_t max_iter, double tol, double* f_out,
                    int32_t* iters_out) {
  if (!c || !c->X || max_iter < 0 || !(tol >= 0.0)) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const int k = c->cfg.k, n = c->cfg.n, npad = c->plan.npad;
  const long long m = c->cfg.m;
  cudaStream_t st = c->stream;
  const int live = count_live_host(c->ws.mask_inc, k, st);
  if (live < 0) return BM_ECUDA;
  if (live == 0) return BM_EINVAL;   // no incumbent yet
  // update-pass shape: one CTA per SM; the widest feature block (up to 256)
  // that leaves room for at least four private warp slices, else one
  const size_t budget = kSmemLimit - 8 * 1024;
  int fw = 0, wu = 0;
  for (int need : {4, 1}) {
    for (int cand : {256, 128, 64, 32}) {
      const int w = std::min(cand, npad);
      int u = 8;
      while (u > need && polish_smem(k, w, u) > budget) --u;
      if (polish_smem(k, w, u) <= budget) { fw = w; wu = u; break; }
    }
    if (fw) break;
  }
  if (fw == 0) return BM_EUNSUPPORTED;
  const size_t psmem = polish_smem(k, fw, wu);
  const int G = sm_count();
  if (!c->pol_labels) {
    if (cudaMalloc(&c->pol_labels, (size_t)m * 4) != cudaSuccess ||
        cudaMalloc(&c->pol_sum, (size_t)G * k * npad * 4) != cudaSuccess ||
        cudaMalloc(&c->pol_cnt, (size_t)G * k * 4) != cudaSuccess)
      return BM_ENOMEM;
    c->pol_grid = G;
  }
  // work on the working copy (C, mask), starting from the incumbent
  if (cudaMemcpyAsync(c->ws.C, c->ws.Cinc, (size_t)k * npad * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->ws.mask, c->ws.mask_inc, k, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return BM_ECUDA;
  PolishArgs pa{};
  pa.X = c->X; pa.m = m; pa.n = n; pa.npad = npad; pa.k = k;
  pa.C = c->ws.C; pa.cstride = npad; pa.mask = c->ws.mask; pa.labels = c->pol_labels;
  pa.part_sum = c->pol_sum; pa.part_cnt = c->pol_cnt;
  pa.rows_per_cta = (m + c->pol_grid - 1) / c->pol_grid;
  pa.wu = wu;
  pa.fw = fw;
  pa.empty_keep = c->cfg.empty == BM_EMPTY_KEEP;
  double f = 0.0, f_prev = 0.0;
  int it = 0;
  while (true) {
    const int nl = count_live_host(c->ws.mask, k, st);
    if (nl <= 0) return nl < 0 ? BM_ECUDA : BM_EINVAL;
    bm_status rc;
    if (c->plan.agrid == 0)
      rc = assign_tc_impl(c->X, m, n, k, c->ws.C, npad, c->ws.mask, c->pol_labels, nullptr,
                          c->ws, st, &f, nullptr, 3, c->plan.cap);
    else
      rc = assign_impl(c->X, m, n, k, c->plan, c->ws.C, npad, c->ws.mask, c->pol_labels,
                       nullptr, c->ws, st, &f);
    if (rc != BM_OK) return rc;
    c->nd_assign += m * (long long)nl;
    const bool stop = (f == 0.0) || (it > 0 && f_prev - f <= tol * f_prev) || (it == max_iter);
    if (launch_polish_update(pa, c->pol_grid, psmem, stop ? 1 : 0, st) != cudaSuccess)
      return BM_ECUDA;
    if (stop) break;
    f_prev = f;
    ++it;
  }
  // the polished centroids become the incumbent (f_opt keeps its sample value)
  if (cudaMemcpyAsync(c->ws.Cinc, c->ws.C, (size_t)k * npad * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->ws.mask_inc, c->ws.mask, k, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return BM_ECUDA;
  if (f_out) *f_out = f;
  if (iters_out) *iters_out = it;
  return BM_OK;
}

bm_status bm_trace(bm_ctx* c, double* ns_out, int32_t count) {
  if (!c || !ns_out || count < 0) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  Stats h{};
  if (cudaMemcpyAsync(&h, c->ws.stats, sizeof(Stats), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return BM_ECUDA;
  for (int i = 0; i < count && i < kNumPhaseTimers; ++i) ns_out[i] = (double)h.phase_ns[i];
  return BM_OK;
}

bm_status bm_get_state(bm_ctx* c, float* C_host, uint8_t* mask_host,
                       double* f_opt, int64_t* chunk_counter) {
  if (!c) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const int k = c->cfg.k, n = c->cfg.n, npad = c->plan.npad;
  cudaStream_t st = c->stream;
  if (C_host &&
      cudaMemcpy2DAsync(C_host, n * 4, c->ws.Cinc, npad * 4, n * 4, k,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BM_ECUDA;
  if (mask_host && cudaMemcpyAsync(mask_host, c->ws.mask_inc, k, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BM_ECUDA;
  if (f_opt && cudaMemcpyAsync(f_opt, c->ws.f_opt, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return BM_ECUDA;
  if (chunk_counter) *chunk_counter = c->t;
  return BM_OK;
}

bm_status bm_objective(bm_ctx* c, double* f_opt_out, float* C_out_host,
                       uint8_t* mask_out_host) {
  return bm_get_state(c, C_out_host, mask_out_host, f_opt_out, nullptr);
}

bm_status bm_set_state(bm_ctx* c, const float* C_host, const uint8_t* mask_host,
                       double f_opt, int64_t chunk_counter) {
  if (!c || !C_host || !mask_host || chunk_counter < 0) return BM_EINVAL;
  std::lock_guard<std::mutex> g(c->mu);
  const int k = c->cfg.k, n = c->cfg.n, npad = c->plan.npad;
  cudaStream_t st = c->stream;
  std::vector<float> pad((size_t)k * npad, 0.f);
  std::vector<uint8_t> m(k);
  for (int j = 0; j < k; ++j) {
    m[j] = mask_host[j] ? 1 : 0;
    for (int f = 0; f < n; ++f) pad[(size_t)j * npad + f] = C_host[(size_t)j * n + f];
  }
  if (cudaMemcpyAsync(c->ws.Cinc, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->ws.mask_inc, m.data(), k, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->ws.f_opt, &f_opt, 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return BM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return BM_ECUDA;
  c->t = chunk_counter;
  return BM_OK;
}

// Device memory of bm_fit_host: a stream-ordered pool per device that keeps
// freed blocks for the next call (held until the process exits), so repeated
// calls neither pay for cudaMalloc nor synchronise the device in cudaFree.

static cudaMemPool_t fit_host_pool(int dev) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> g(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = UINT64_MAX;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

// The device address of host memory the GPU can read directly (pinned or
// registered), or null (pageable memory, or no such mapping).
static const float* host_rows_on_device(const float* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  return static_cast<const float*>(at.devicePointer);
}

bm_status bm_fit_host(const bm_config* cfg, const float* X_host, int32_t chunks,
                      float* C_out_host, uint8_t* mask_out_host,
                      int32_t* labels_out_host, double* sse_out,
                      bm_fit_report* report) {
  if (!cfg || !X_host || chunks < 0) return BM_EINVAL;
  if (!shape_ok(cfg->m, cfg->n, cfg->k, cfg->s)) return BM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return BM_ECUDA; }
  cudaMemPool_t pool = fit_host_pool(dev);
  if (!pool) return BM_ECUDA;
  cudaStream_t st = nullptr, cs = nullptr;
  cudaEvent_t e_alloc = nullptr, e_copied = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return BM_ECUDA;
  float* X = nullptr;
  int32_t* labels = nullptr;
  uint32_t* ready = nullptr;
  const size_t xbytes = (size_t)cfg->m * cfg->n * 4;
  // Rows the GPU can read in place: the copy to the device runs on a second
  // stream while the first chunks gather their samples from host memory;
  // the final assignment waits for the copy.
  const float* Xh = host_rows_on_device(X_host);
  int x_shift = 0;   // the copy pieces' block size, 2^x_shift rows
  bm_status rc = BM_OK;
  bm_ctx* c = nullptr;
  if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&X), xbytes, pool, st) != cudaSuccess) {
    cudaGetLastError();
    rc = BM_ENOMEM;
    goto done;
  }
  if (labels_out_host &&
      cudaMallocFromPoolAsync(reinterpret_cast<void**>(&labels), (size_t)cfg->m * 4, pool, st) !=
          cudaSuccess) {
    cudaGetLastError();
    rc = BM_ENOMEM;
    goto done;
  }
  if (Xh) {
    if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ready), 16, pool, st) != cudaSuccess ||
        cudaMemsetAsync(ready, 0, 16, st) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e_alloc, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e_copied, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(e_alloc, st) != cudaSuccess ||
        cudaStreamWaitEvent(cs, e_alloc, 0) != cudaSuccess) {
      rc = BM_ECUDA;
      goto done;
    }
    // the copy in kHostCopyPieces interleaved pieces, each followed by the
    // count of pieces landed so far: X is cut into blocks of 2^x_shift rows
    // and piece p takes blocks p, p + P, p + 2P, ... (one strided copy), so
    // every CTA's share of a chunk's sorted sample -- a 1/G slice of the
    // rows -- spans all pieces and moves to the device copy at the same pace
    // (with pieces of consecutive rows, the CTAs holding the last rows read
    // all of theirs from host memory until the copy reached them, and every
    // chunk waited for those CTAs).  Blocks: at most m / 4096 rows, so a
    // slice of the rows spans every piece, and strides below 1 GB.
    const size_t rowb = (size_t)cfg->n * 4;
    const long long P = kHostCopyPieces;
    x_shift = 0;
    while ((2LL << x_shift) <= cfg->m / 4096 &&
           (size_t)P * ((size_t)2 << x_shift) * rowb <= ((size_t)1 << 30))
      ++x_shift;
    const long long B = 1LL << x_shift, nfull = cfg->m >> x_shift;   // full blocks
    const size_t bbytes = (size_t)B * rowb;
    char* Xd = reinterpret_cast<char*>(X);
    const char* Xs = reinterpret_cast<const char*>(X_host);
    for (long long p = 0; p < P && rc == BM_OK; ++p) {
      cudaError_t e = cudaSuccess;
      const long long h = nfull > p ? (nfull - 1 - p) / P + 1 : 0;   // full blocks p + P j
      if (h > 0)
        e = cudaMemcpy2DAsync(Xd + (size_t)p * bbytes, (size_t)P * bbytes, Xs + (size_t)p * bbytes,
                              (size_t)P * bbytes, bbytes, (size_t)h, cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess && nfull % P == p && (cfg->m & (B - 1)) != 0) {   // the last, partial block
        const size_t off = (size_t)nfull * bbytes, len = (size_t)(cfg->m - nfull * B) * rowb;
        e = cudaMemcpyAsync(Xd + off, Xs + off, len, cudaMemcpyHostToDevice, cs);
      }
      if (e != cudaSuccess || launch_x_ready(ready, (uint32_t)(p + 1), cs) != cudaSuccess)
        rc = BM_ECUDA;
    }
    if (rc != BM_OK || cudaEventRecord(e_copied, cs) != cudaSuccess) {
      rc = BM_ECUDA;
      goto done;
    }
  } else if (cudaMemcpyAsync(X, X_host, xbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    rc = BM_ECUDA;
    goto done;
  }
  {
    // a one-shot context: recording a graph would not pay for itself; its
    // workspace comes from the same pool
    bm_config once = *cfg;
    once.graphs = 0;
    rc = bm::ctx_create(&once, X, st, pool, &c, 0);
  }
  if (rc != BM_OK) goto done;
  if (Xh) {
    c->Xh = Xh;
    c->x_ready = ready;
    c->x_shift = x_shift;
  }
  rc = bm_fit_chunk(c, chunks, report);
  if (Xh) {
    c->Xh = nullptr;
    c->x_ready = nullptr;
    if (cudaStreamWaitEvent(st, e_copied, 0) != cudaSuccess && rc == BM_OK) rc = BM_ECUDA;
  }
  if (rc != BM_OK) goto done;
  rc = bm_assign(c, labels, sse_out);
  if (rc != BM_OK) goto done;
  if (labels_out_host &&
      (cudaMemcpyAsync(labels_out_host, labels, (size_t)cfg->m * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess)) { rc = BM_ECUDA; goto done; }
  rc = bm_objective(c, nullptr, C_out_host, mask_out_host);
done:
  // the copy (and the flag write after it) ends before X and the flag go
  if (cs) cudaStreamSynchronize(cs);
  if (c) bm_destroy(c);
  if (ready) cudaFreeAsync(ready, st);
  if (labels) cudaFreeAsync(labels, st);
  if (X) cudaFreeAsync(X, st);
  cudaStreamSynchronize(st);
  if (e_alloc) cudaEventDestroy(e_alloc);
  if (e_copied) cudaEventDestroy(e_copied);
  if (cs) cudaStreamDestroy(cs);
  cudaStreamDestroy(st);
  return rc;
}

// ------------------------------------------------------------ step level
// Each call builds a private workspace, runs, and frees it.
static std::mutex g_ops_mu;

bm_status bm_draw_chunk(int64_t m, int64_t s, uint64_t seed, int64_t t,
                        int32_t* idx_dev, void* stream) {
  if (!idx_dev || !shape_ok(m, 1, 1, s) || t < 0) return BM_EINVAL;
  std::lock_guard<std::mutex> g(g_ops_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* bitmap = nullptr;
  const size_t words = draw_bitmap_words(m);
  if (cudaMalloc(&bitmap, words * 4) != cudaSuccess) return BM_ENOMEM;
  bm_status rc = BM_OK;
  if (cudaMemsetAsync(bitmap, 0, words * 4, st) != cudaSuccess) rc = BM_ECUDA;
  DrawArgs d{};
  d.m = m; d.s = (int)s; d.seed = seed; d.t0 = t; d.idx = idx_dev; d.bitmaps = bitmap;
  if (rc == BM_OK && launch_draw(d, 1, st) != cudaSuccess) rc = BM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = BM_ECUDA;
  cudaFree(bitmap);
  return rc;
}

bm_status bm_gather(const float* X_dev, int64_t m, int32_t n,
                    const int32_t* idx_dev, int64_t s, float* P_dev,
                    void* stream) {
  if (!X_dev || !idx_dev || !P_dev || !shape_ok(m, n, 1, s)) return BM_EINVAL;
  std::lock_guard<std::mutex> g(g_ops_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan p;
  bm_status rc = make_plan(n, 1, s, &p);
  if (rc != BM_OK) return rc;
  Workspace w;
  rc = ws_create(&w, m, 1, s, p, st);
  if (rc != BM_OK) return rc;
  ChunkArgs a = chunk_args(w, p, X_dev, m, n, 1, s);
  a.idx = const_cast<int32_t*>(idx_dev);
  a.phases = kPhaseGather;
  if (launch_plan(a, p, st) != cudaSuccess) rc = BM_ECUDA;
  if (rc == BM_OK) rc = check_status(w, st, m);
  if (rc == BM_OK &&
      cudaMemcpy2DAsync(P_dev, n * 4, w.P, p.npad * 4, n * 4, s, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    rc = BM_ECUDA;
  cudaStreamSynchronize(st);
  w.release();
  return rc;
}

// Copies P (s x n) and (C, mask) into a fresh workspace with padded rows.
static bm_status stage_inputs(Workspace& w, const Plan& p, const float* P_dev,
                              long long s, int n, int k, const float* C_dev,
                              const uint8_t* mask_dev, cudaStream_t st) {
  if (cudaMemsetAsync(w.P, 0, (size_t)s * p.npad * 4, st) != cudaSuccess) return BM_ECUDA;
  if (cudaMemcpy2DAsync(w.P, p.npad * 4, P_dev, n * 4, n * 4, s, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return BM_ECUDA;
  if (cudaMemcpy2DAsync(w.C, p.npad * 4, C_dev, n * 4, n * 4, k, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return BM_ECUDA;
  if (cudaMemcpyAsync(w.mask, mask_dev, k, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return BM_ECUDA;
  return BM_OK;
}

static bm_status unstage_outputs(Workspace& w, const Plan& p, int n, int k,
                                 float* C_dev, uint8_t* mask_dev, cudaStream_t st) {
  if (cudaMemcpy2DAsync(C_dev, n * 4, w.C, p.npad * 4, n * 4, k, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return BM_ECUDA;
  if (cudaMemcpyAsync(mask_dev, w.mask, k, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return BM_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? BM_OK : BM_ECUDA;
}

bm_status bm_kpp_reseed(const float* P_dev, int64_t s, int32_t n, int32_t k,
                        float* C_dev, uint8_t* mask_dev, uint64_t seed,
                        int64_t t, int32_t trials, void* stream) {
  if (!P_dev || !C_dev || !mask_dev || !shape_ok(s, n, k, s) || t < 0 ||
      trials < 1 || trials > kMaxTrials)
    return BM_EINVAL;
  std::lock_guard<std::mutex> g(g_ops_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan p;
  bm_status rc = make_plan(n, k, s, &p);
  if (rc != BM_OK) return rc;
  Workspace w;
  rc = ws_create(&w, s, k, s, p, st);
  if (rc != BM_OK) return rc;
  rc = stage_inputs(w, p, P_dev, s, n, k, C_dev, mask_dev, st);
  ChunkArgs a = chunk_args(w, p, nullptr, s, n, k, s);
  a.seed = seed;
  a.t = t;
  a.trials = trials;
  a.phases = kPhaseKpp;
  if (rc == BM_OK && launch_plan(a, p, st) != cudaSuccess) rc = BM_ECUDA;
  if (rc == BM_OK) rc = check_status(w, st, s);
  if (rc == BM_OK) rc = unstage_outputs(w, p, n, k, C_dev, mask_dev, st);
  cudaStreamSynchronize(st);
  w.release();
  return rc;
}

bm_status bm_lloyd(const float* P_dev, int64_t s, int32_t n, int32_t k,
                   float* C_dev, uint8_t* mask_dev, int32_t max_iter,
                   double tol, double* f_out, int32_t* iters_out,
                   void* stream) {
  if (!P_dev || !C_dev || !mask_dev || !shape_ok(s, n, k, s) || max_iter < 0 ||
      !(tol >= 0.0))
    return BM_EINVAL;
  std::lock_guard<std::mutex> g(g_ops_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (count_live_host(mask_dev, k, st) <= 0) return BM_EINVAL;
  Plan p;
  bm_status rc = make_plan(n, k, s, &p);
  if (rc != BM_OK) return rc;
  Workspace w;
  rc = ws_create(&w, s, k, s, p, st);
  if (rc != BM_OK) return rc;
  rc = stage_inputs(w, p, P_dev, s, n, k, C_dev, mask_dev, st);
  ChunkArgs a = chunk_args(w, p, nullptr, s, n, k, s);
  a.max_iter = max_iter;
  a.tol = tol;
  a.phases = kPhaseLloyd;
  if (rc == BM_OK && launch_plan(a, p, st) != cudaSuccess) rc = BM_ECUDA;
  if (rc == BM_OK) rc = check_status(w, st, s);
  if (rc == BM_OK) rc = unstage_outputs(w, p, n, k, C_dev, mask_dev, st);
  if (rc == BM_OK) {
    Ctl h{};
    if (cudaMemcpy(&h, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) rc = BM_ECUDA;
    if (f_out) *f_out = h.f_out;
    if (iters_out) *iters_out = h.iters_out;
  }
  cudaStreamSynchronize(st);
  w.release();
  return rc;
}

bm_status bm_assign_rows_prec(const float* X_dev, int64_t m, int32_t n,
                              const float* C_dev, const uint8_t* mask_dev,
                              int32_t k, int32_t precision, int32_t* labels_dev,
                              float* dmin_dev, double* sse_out,
                              uint64_t* rescored_out, void* stream) {
  if (precision == BM_FP32) {
    if (rescored_out) *rescored_out = 0;
    return bm_assign_rows(X_dev, m, n, C_dev, mask_dev, k, labels_dev, dmin_dev, sse_out,
                          stream);
  }
  if (precision != BM_BF16_RESCORE && precision != BM_BF16X3_RESCORE &&
      precision != BM_FP8_RESCORE)
    return BM_EUNSUPPORTED;
  if (!X_dev || !C_dev || !mask_dev || m < 1 || n < 1 || k < 1 || m > 2147483647LL)
    return BM_EINVAL;
  std::lock_guard<std::mutex> g(g_ops_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (count_live_host(mask_dev, k, st) <= 0) return BM_EINVAL;
  Plan p;   // only the assignment scratch is used: a minimal chunk plan
  bm_status rc = make_plan(1, 1, 1, &p);
  if (rc != BM_OK) return rc;
  Workspace w;
  rc = ws_create(&w, 1, 1, 1, p, st, 1, m);
  if (rc != BM_OK) return rc;
  unsigned long long resc = 0;
  rc = assign_tc_impl(X_dev, m, n, k, C_dev, n, mask_dev, labels_dev, dmin_dev, w, st,
                      sse_out, &resc, assign_terms(precision));
  if (rescored_out) *rescored_out = resc;
  cudaStreamSynchronize(st);
  w.release();
  return rc;
}

bm_status bm_assign_rows(const float* X_dev, int64_t m, int32_t n,
                         const float* C_dev, const uint8_t* mask_dev,
                         int32_t k, int32_t* labels_dev, float* dmin_dev,
                         double* sse_out, void* stream) {
  if (!X_dev || !C_dev || !mask_dev || m < 1 || n < 1 || k < 1 || m > 2147483647LL)
    return BM_EINVAL;
  std::lock_guard<std::mutex> g(g_ops_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (count_live_host(mask_dev, k, st) <= 0) return BM_EINVAL;
  Plan p;
  bm_status rc = make_plan(n, k, std::max<long long>(k, 1), &p);
  if (rc != BM_OK) return rc;
  Workspace w;
  rc = ws_create(&w, k, k, k, p, st, 1, p.agrid == 0 ? m : 0);
  if (rc != BM_OK) return rc;
  if (p.agrid == 0)
    rc = assign_tc_impl(X_dev, m, n, k, C_dev, n, mask_dev, labels_dev, dmin_dev, w, st,
                        sse_out, nullptr, 3);
  else
    rc = assign_impl(X_dev, m, n, k, p, C_dev, n, mask_dev, labels_dev, dmin_dev, w, st, sse_out);
  cudaStreamSynchronize(st);
  w.release();
  return rc;
}

}  // extern "C"
