// Internal declarations shared by the host driver and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace bm {

constexpr int kMaxTrials = 4;      // K-means++ candidates per centre (paper: 3)
constexpr int kMaxK = 128;         // centroids per job handled by the kernels
constexpr int kRoundSlots = 64;    // per-round draw counters (== kMaxRounds)
constexpr int kNpMax = 32;         // widest row kept in registers

// Phases of the chunk kernel (Alg. 1 loop body).
enum Phase : int {
  kPhaseDraw = 1,     // sample indices of chunk t
  kPhaseGather = 2,   // P = X[idx]
  kPhaseKpp = 4,      // K-means++ reseed of degenerate centroids
  kPhaseLloyd = 8,    // K-means on P
  kPhaseKeep = 16,    // keep-the-best against the incumbent
};

// Device control block of one workspace.  Zeroed at creation; every launch
// leaves it ready for the next one (see the kernel epilogue).
struct Ctl {
  uint32_t bar[2];                    // alternating grid-barrier counters
  uint32_t round_cnt[kRoundSlots];    // new distinct draws per sample round
  int32_t status;                     // sticky error word (bm_status values)
  int32_t cand[kMaxTrials];           // K-means++ candidate rows of a slot
  int32_t iters_out;                  // Lloyd update steps of the last launch
  double f_out;                       // f(C'', P) of the last launch
  uint32_t assign_ticket;             // last-CTA ticket of the assign kernel
  uint32_t pad_;
};

// Cumulative counters of a context, updated on the device by CTA 0.
struct Stats {
  long long chunks;
  long long accepted;
  long long lloyd_iters;
  long long n_d;
};

struct ChunkArgs {
  const float* X;      // m x n (row stride n)
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
  int kpad;            // k rounded up to 32 (generic path)
  int32_t* idx;        // s
  uint32_t* bitmap;    // ceil(m / 32), all zero between launches
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
};

// Shared-memory layout of the chunk kernel (bytes), identical on host/device.
struct ChunkSmem {
  int cen, live, sw, cw, lab, dmin, dc, cand, stage, red, total;
  int wu;              // warps that own an update slice
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline ChunkSmem chunk_smem(int npad, int k, int kpad, int R,
                                                bool generic) {
  ChunkSmem L;
  int o = 0;
  L.cen = o;   o += align_up((generic ? npad * kpad : k * npad) * 4, 16);
  L.live = o;  o += align_up(k * 4, 16);
  // update slices: as many warps as fit in 64 KB (at least one)
  int per = k * 32 * 4;
  int wu = (64 * 1024) / per;
  if (wu > 8) wu = 8;
  if (wu < 1) wu = 1;
  L.wu = wu;
  L.sw = o;    o += align_up(wu * per, 16);
  L.cw = o;    o += align_up(wu * k * 4, 16);
  L.lab = o;   o += align_up(R * 4, 16);
  L.dmin = o;  o += align_up(R * 4, 16);
  L.dc = o;    o += align_up(kMaxTrials * R * 4, 16);
  L.cand = o;  o += align_up(kMaxTrials * npad * 4, 16);
  L.stage = o; o += generic ? align_up(64 * npad * 4, 16) : 0;
  L.red = o;   o += 64 * 8;
  L.total = o;
  return L;
}

// Host-side launch helpers (bm_kernels.cu).
cudaError_t launch_chunk(const ChunkArgs& a, int grid, bool generic, int np,
                         size_t smem, cudaStream_t st);
int chunk_max_grid(bool generic, int np, size_t smem);
cudaError_t launch_assign(const AssignArgs& a, int grid, bool generic, int np,
                          size_t smem, cudaStream_t st);
int assign_max_grid(bool generic, int np, size_t smem);
size_t assign_smem(int npad, int k, int kpad, bool generic);

}  // namespace bm
