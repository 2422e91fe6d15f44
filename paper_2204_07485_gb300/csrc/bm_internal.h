// Internal declarations shared by the host driver and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bigmeans.h"

namespace bm {

constexpr int kMaxTrials = 4;      // K-means++ candidates per centre (paper: 3)
constexpr int kMaxK = 128;         // centroids per job handled by the kernels
constexpr int kTermsFp8 = 8;       // AssignTcArgs::terms of the E4M3 form
constexpr int kRoundSlots = 64;    // per-round draw counters (== kMaxRounds)
constexpr int kNpMax = 32;         // widest row kept in registers
constexpr int kNumPhaseTimers = 11;
// Pieces of bm_fit_host's host-to-device copy of X (a power of two: a row's
// piece is its block index modulo this).
constexpr int kHostCopyPieces = 32;
static_assert((kHostCopyPieces & (kHostCopyPieces - 1)) == 0, "pieces: a power of two");  // see Stats::phase_ns

// Reinitialisation of degenerate centroids (bm_config.init).
constexpr int kInitKmeanspp = 0;
constexpr int kInitForgy = 1;

// Phases of the chunk kernel (Alg. 1 loop body).
enum Phase : int {
  kPhaseGather = 2,   // P = X[idx] (idx drawn ahead by the sample plan)
  kPhaseKpp = 4,      // K-means++ reseed of degenerate centroids
  kPhaseLloyd = 8,    // K-means on P
  kPhaseKeep = 16,    // keep-the-best against the incumbent
};

// Device control block of one workspace.  Zeroed at creation; every launch
// leaves it ready for the next one (see the kernel epilogue).
struct Ctl {
  uint32_t bar[2];                    // alternating grid-barrier counters
  int32_t status;                     // sticky error word (bm_status values)
  int32_t cand[kMaxTrials];           // K-means++ candidate rows of a slot
  int32_t iters_out;                  // Lloyd update steps of the last launch
  double f_out;                       // f(C'', P) of the last launch
  uint32_t assign_ticket;             // last-CTA ticket of the assign kernel
  uint32_t late;                      // K-means++ exchange reads that found their
                                      // value not yet published (see bm_kpp.cuh)
};

// Cumulative counters of a context, updated on the device by CTA 0.
struct Stats {
  long long chunks;
  long long accepted;
  long long lloyd_iters;
  long long n_d;
  // device time per phase (ns, CTA 0's %globaltimer between its phase
  // boundaries): [0] setup, [1] gather, [2] K-means++, [3] Lloyd own rows
  // (assignment + partial sums), [4] Lloyd first barrier wait, [5] Lloyd
  // cross-CTA reduction + update, [6] Lloyd second barrier wait + reload,
  // [7] keep-the-best; [8..10] split [3] into assignment, update slices and
  // slice combination + partial-sum stores
  unsigned long long phase_ns[kNumPhaseTimers];
  long long host_gathers;   // CTA gathers made while part of X was still only in host memory
};

struct ChunkArgs {
  const float* X;      // m x n (row stride n)
  // Optional second copy of X in device-accessible host memory: while X is
  // being filled by a host-to-device copy in kHostCopyPieces interleaved
  // pieces (blocks of 2^x_shift rows, block b in piece b mod
  // kHostCopyPieces, pieces landing in order), *x_ready counts the pieces
  // that have landed; a gather reads a row from X when its piece has landed
  // and from Xh otherwise.  Both hold the same bytes.  Null: X only.
  const float* Xh;
  const uint32_t* x_ready;
  int x_shift;
  long long m;
  int n, npad, k, s;
  int rows_per_cta;    // R = ceil(s / gridDim.x)
  unsigned long long seed;
  long long t;         // chunk index
  int max_iter;
  double tol;
  int trials;
  int phases;
  int bar_sel;         // which Ctl::bar counter this launch uses
  int trace;           // 1: CTA 0 times its phases into Stats::phase_ns
  int init;            // reinitialisation of degenerate centroids: kInitKmeanspp / kInitForgy
  int empty_keep;      // 1: a centroid without members keeps its position, live
  int kpad;            // k rounded up to 32 (generic path)
  int32_t* idx;        // s
  float* P;            // s x npad
  float* C;            // k x npad working centroids (C', C'')
  uint8_t* mask;       // k working mask
  float* Cinc;         // k x npad incumbent
  uint8_t* mask_inc;   // k
  double* f_opt;       // incumbent objective
  float* part_sum;     // [k][npad][G]
  int32_t* part_cnt;   // [k][G]
  double* part_f;      // [kMaxTrials][G]
  int32_t* blk_cnt;    // [G]
  Ctl* ctl;
  Stats* stats;
  // K-means++ exchange tags (bm_kpp.cuh): [0] the launch generation, then
  // [1, 1 + G) the D^2 block sums', [1 + G, 1 + 2G) the potentials' and
  // [1 + 2G, 1 + 2G + kMaxTrials) the candidate rows' tags
  unsigned long long* kx;
  // tensor-core chunk kernel (rows wider than 32 features)
  int tc_kb;              // K blocks of 128-byte rows: 64 BF16 or 128 E4M3 features
  int tc_n16;             // MMA N: k rounded up to 16
  int tc_ncols;           // TMEM columns
  int tc_fb;              // features per staged block of the exact passes
  int tc_tpc;             // 128-row tiles per CTA: ceil(rows_per_cta / 128)
  int tc_ns;              // MMA ring slots (2 or 3)
  int tc_planes;          // planes of the screening products: 1 (BF16 or E4M3) or
                          // 2 (split BF16: hi*hi + hi*lo + lo*hi)
  int tc_fp8;             // 1: E4M3 screening (rows scaled per row, centroids by
                          // one power of two per chunk), tc_planes = 1
  unsigned char* Cb;      // BF16: [tc_kb][2][tc_n16][128 B] centroid planes (hi, lo);
                          // E4M3: [tc_kb][tc_n16][128 B]; swizzled
  float* sqs;             // [k][ceil(npad / 8)] squared norms of 8-feature slices of C
  unsigned char* Pb;      // [G][tc_tpc][tc_kb][tc_planes][128][128 B] own-row planes, swizzled
};

struct AssignArgs {
  const float* X;      // m x n, row stride n
  long long m;
  int n, npad, k, kpad;
  const float* C;      // k x cstride
  int cstride;
  const uint8_t* mask; // k
  int32_t* labels;     // m or null
  float* dmin;         // m or null
  double* part;        // [G]
  double* sse;         // device scalar
  uint32_t* ticket;    // zero between launches
  int* status;         // debug builds: index-guard status word (may be null)
};

// Words of one chunk's bitmap in global memory: ceil(m / 32) rounded up to a
// multiple of four, so every chunk's bitmap starts on a 16-byte boundary.
__host__ __device__ inline size_t draw_bitmap_words(long long m) {
  return (size_t)(((m + 31) / 32 + 3) / 4 * 4);
}

struct DrawArgs {
  long long m;
  int s;
  unsigned long long seed;
  long long t0;        // first chunk of the batch; CTA b draws chunk t0 + b
  int32_t* idx;        // [batch][s] sorted sample rows
  uint32_t* bitmaps;   // [batch][draw_bitmap_words(m)], all zero between launches
  int smem_bitmap;     // set by launch_draw: the bitmap fits in shared memory
  int* status;         // debug builds: index-guard status word (may be null)
};

struct AssignTcArgs {
  const float* X;      // m x n, row stride n
  long long m;
  int n;
  const float* C;      // k x cstride
  int cstride;
  const uint8_t* mask; // k
  int k;
  int32_t* labels;     // m or null
  float* dmin;         // m or null
  float2* part;        // [ceil(m / 128)] per-tile SSE as (hi, lo) pairs
  double* sse;         // device scalar
  uint32_t* ticket;    // zero between launches
  unsigned long long* rescored;  // rows that needed exact rechecks (added to)
  int* status;         // BM_ETIMEOUT when a bounded wait gave up
  int kb;              // K blocks of 64 BF16
  int npad16;          // MMA N: k rounded up to 16 (<= 128)
  int ncols;           // TMEM columns allocated
  int stages;          // FP32 row tiles filled ahead by bulk copies (0: thread loads)
  int use_bulk;        // X is 16-byte aligned: bulk copies for full tiles
  int terms;           // 1: BF16 products; 3: split BF16 (hi*hi + hi*lo + lo*hi);
                       // kTermsFp8: E4M3 products of power-of-two scaled operands
  int cf;              // FP32 centroid copy kept in shared memory
};

// Full-data Lloyd update (bm_polish): per-CTA partials over fixed row ranges.
struct PolishArgs {
  const float* X;          // m x n, row stride n
  long long m;
  int n, npad, k;
  float* C;                // k x cstride working centroids (updated in place)
  int cstride;
  uint8_t* mask;           // k live flags (cleared for centroids without members,
                           // unless empty_keep)
  int empty_keep;          // 1: a centroid without members keeps its position, live
  const int32_t* labels;   // m labels of the last assignment
  float* part_sum;         // [G][k][npad]
  int32_t* part_cnt;       // [G][k]
  long long rows_per_cta;
  int wu;                  // warps with a private slice
  int f0, fw;              // feature block of one update pass (fw <= 256)
};

// Shared-memory layout of the chunk kernel (bytes), identical on host/device.
struct ChunkSmem {
  int cen, crow, live, lidx, sw, cw, lab, dmin, dc, cand, stage, prow, red, total;
  int wu;              // tiled path: row groups that own a private update accumulator
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Register row width of the row-in-register kernels for n <= kNpMax.
__host__ __device__ inline int np_width(int n) {
  return n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : n <= 28 ? 28 : 32;
}

// Threads per CTA of the chunk kernel: 384 for the row-in-register path
// (one sample row per thread for up to 384 rows per CTA, leaving up to 170
// registers per thread), 256 for the tiled path.
__host__ __device__ inline int chunk_threads(bool generic) { return generic ? 256 : 384; }

__host__ __device__ inline ChunkSmem chunk_smem(int npad, int k, int kpad, int R,
                                                bool generic) {
  ChunkSmem L;
  int o = 0;
  const int nthreads = chunk_threads(generic);
  L.cen = o;   o += align_up((generic ? npad * kpad : k * npad) * 4, 16);
  L.crow = o;  o += generic ? align_up(k * npad * 4, 16) : 0;   // row-major copy
  L.live = o;  o += align_up(k * 4, 16);
  L.lidx = o;  o += align_up((k + 1) * 4, 16);   // live list, count at [k]
  int wu = 1;
  if (generic) {
    // one [k][npad] accumulator per row group, threads = groups x features
    wu = nthreads / npad;
    const int cap = (64 * 1024) / (k * npad * 4);
    if (wu > cap) wu = cap;
    if (wu > 8) wu = 8;
    if (wu < 1) wu = 1;
  }
  L.wu = wu;
  // tiled path: update accumulators [wu][k][npad] and counts [wu][k];
  // row-in-register path: the label sort -- order[R], start[k + 1], cur[k]
  // -- and per-warp label counts [warps][k]
  L.sw = o;    o += align_up((generic ? wu * k * npad : R + 2 * k + 1) * 4, 16);
  L.cw = o;    o += align_up((generic ? wu : nthreads / 32) * k * 4, 16);
  L.lab = o;   o += align_up(R * 4, 16);
  L.dmin = o;  o += align_up(R * 4, 16);
  L.dc = o;    o += align_up(kMaxTrials * R * 4, 16);
  L.cand = o;  o += align_up(kMaxTrials * npad * 4, 16);
  L.stage = o; o += generic ? align_up(64 * npad * 4, 16) : 0;
  // row-in-register path: the CTA's R sample rows stay resident for the chunk
  L.prow = o;  o += generic ? 0 : align_up(R * npad * 4, 16);
  L.red = o;   o += 80 * 8;
  L.total = o;
  return L;
}

// Lets launches of fn use up to the device's opt-in shared memory (minus the
// kernel's static shared memory).  Every caller sets the same value, so
// threads preparing launches of different sizes at once cannot lower the
// limit under each other's feet (setting the launch's own size would).
template <typename Kernel>
inline cudaError_t allow_max_smem(Kernel fn) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

// Cooperative launch (all CTAs co-resident, as the grid barriers need) through
// the launch-attribute API, which stream capture records into a graph.
template <typename Kernel>
inline cudaError_t launch_cooperative(Kernel fn, int grid, int threads, size_t smem,
                                      cudaStream_t st, const ChunkArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, a);
}

// Host-side launch helpers (bm_kernels.cu, bm_sample.cu, bm_tc.cu).
cudaError_t launch_draw(const DrawArgs& a, int chunks, cudaStream_t st);
// *landed <- max(*landed, count) once every earlier operation of the stream
// has completed (the pieces of the host-to-device copy of X before it).
cudaError_t launch_x_ready(uint32_t* landed, uint32_t count, cudaStream_t st);
// Streaming tensor-core final assignment (n <= 128, n % 4 == 0, k <= 128):
// shared memory of its plan, 0 when it does not take the shape.
struct TcsPlan {
  int w;        // compute warpgroups
  int na;       // A-tile buffers
  int stages;   // 16 KB column boxes in flight
  int ncols;    // TMEM columns allocated
};
size_t assign_tcs_plan(int n, int k, int terms, size_t limit, TcsPlan* out);
cudaError_t launch_assign_tcs(const float* X, long long m, int n, const float* C, int cstride,
                              const uint8_t* mask, int k, int32_t* labels, float* dmin,
                              float2* part, double* sse, uint32_t* ticket,
                              unsigned long long* rescored, int* status, int terms,
                              const TcsPlan& plan, size_t smem, int grid, cudaStream_t st);
size_t assign_tc_smem(int n, int k, int terms, int* stages, int* kb, int* npad16,
                      int* ncols, int* cf, bool bulk_ok, size_t limit);
int assign_tc_max_grid(size_t smem, int terms);
cudaError_t launch_assign_tc(const AssignTcArgs& a, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_chunk(const ChunkArgs& a, int grid, bool generic, int np,
                         size_t smem, cudaStream_t st);
// tensor-core chunk kernel: shared memory for (npad, k, R, n16, fb, ring
// slots); CTAs that can be co-resident; launch
size_t chunk_tc_smem(int npad, int k, int R, int n16, int fb, int ns, int planes);
int chunk_tc_max_grid(size_t smem);
cudaError_t launch_chunk_tc(const ChunkArgs& a, int grid, size_t smem, cudaStream_t st);
size_t polish_smem(int k, int fw, int wu);
cudaError_t launch_polish_update(const PolishArgs& a, int grid, size_t smem, int stop,
                                 cudaStream_t st);
int chunk_max_grid(bool generic, int np, size_t smem);
cudaError_t launch_assign(const AssignArgs& a, int grid, bool generic, int np,
                          size_t smem, cudaStream_t st);
int assign_max_grid(bool generic, int np, size_t smem);
size_t assign_smem(int npad, int k, int kpad, bool generic);

}  // namespace bm

// Context construction shared by bm_create and the job server: allocations
// from `pool` (stream-ordered on `stream`) when it is not null; and the
// device bytes a context for cfg would hold.
namespace bm {
bm_status ctx_create(const bm_config* cfg, const float* X_dev, cudaStream_t stream,
                     cudaMemPool_t pool, bm_ctx** out, int plan_cap = 0);
bm_status ctx_footprint(const bm_config* cfg, size_t* bytes);
}  // namespace bm
