// Grouped Lloyd: many independent Lloyd problems (Sec. 2, stop rule of
// Sec. 5) advanced together, one launch per Lloyd step for all of them
// (bm_group_create / bm_group_run / bm_group_destroy).
//
// Work layout.  Every problem's rows form 64-row tiles; the tiles of all
// problems, problem after problem, form one list, and the list is cut into
// one contiguous range per CTA of equal estimated cost (a tile of problem p
// costs about n_p * (ceil(k_p / 32) + 1)), so a large problem spreads over
// many SMs and small ones share an SM.  The part of a CTA's range that lies
// in one problem is a segment; a segment owns a slot of partial results.
//
//   group_step_kernel  (one cooperative launch per Lloyd step)
//     assignment: per segment of an unfinished problem: the problem's
//     centroids into shared memory, then per tile the nearest live centroid
//     of each row (FP32 direct differences summed over features in order,
//     lowest index on ties), the row's label, and the row's (x - c_label)
//     added into per-row-group accumulators in a fixed row order; at the end
//     the segment's sums, member counts and objective go to its slot;
//     a grid barrier;
//     update: CTA b takes problems b, b + G, ...: the problem's slots added
//     in CTA order (the objective in float64), the stop test, degenerate
//     marking of live centroids without members, the centroid update unless
//     stopping, and the problem's state.
//   (group_assign_kernel + group_update_kernel: the same two phases as two
//   launches, for a grid that cannot be co-resident -- one CTA per problem
//   beyond the GPU's capacity -- and for the tile autotuner.)
//
// Tile shapes.  A 64-row tile's distances are computed either with one lane
// per centroid (8 rows per warp, centroids in groups of 32) or, for k <= 16,
// with four lanes per row (each lane a quarter of the centroids), which
// keeps lanes busy when k is small.  Both add the same squared differences
// in the same order and settle ties the same way, and the row's distance is
// credited to the same thread, so the shape changes no bit of the results.
// On its first run a group times both shapes on the problems of each (n, k)
// with k <= 16 and keeps the faster (bm_group_set_tiles can fix a shape).
//
// A CUDA graph of a few steps is recorded once and replayed until no
// problem is left; finished problems cost a flag test per segment, and after
// a replay that finished some problems the tile list of the others is cut
// again over all CTAs (the tables live in device memory, so the recorded
// graph stays valid).  Every sum has a fixed order and the partitions depend
// only on the data, so results are reproducible.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_device.cuh"
#include "bm_internal.h"
#include "bm_tile.cuh"

namespace bm {

constexpr int kGroupThreads = 256;   // nearest_tile: 8 warps x 8 rows
constexpr int kGroupStepsPerGraph = 2;
constexpr size_t kGroupSmemLimit = 227 * 1024;

struct GroupProb {
  const float* P;
  float* C;
  uint8_t* mask;
  int* labels;
  long long s;
  int n, npad, k, kpad;
  int ng;            // row groups with private accumulators
  int slot0, slot1;  // the problem's slots [slot0, slot1), in CTA order
  int rows_tile;     // tile shape: 0 = a lane per centroid, 1 = four lanes per row (k <= 16)
};

struct GroupSeg {
  int prob;
  int t0, t1;        // tiles [t0, t1) of the problem
};

struct GroupSlotOff {
  long long sum;     // offset of the slot's [k][npad] sums (floats)
  long long cnt;     // offset of the slot's [k] counts (ints)
};

struct GroupState {
  double f, f_prev;
  long long nd;      // point-centroid distance evaluations
  int it, done, live, pad;
};

struct GroupArgs {
  const GroupProb* probs;
  const GroupSeg* segs;       // slot i = segment i
  const GroupSlotOff* offs;
  const int* cta_seg;         // CTA c: segments [cta_seg[c], cta_seg[c + 1])
  float* part_sum;
  int* part_cnt;
  double* part_f;
  GroupState* st;
  int* active;                // unfinished problems
  int count, max_iter;
  double tol;
  int npad_max, kpad_max, acc_floats;   // shared-memory layout
  uint32_t* bar;              // [2] grid-barrier counters of the step kernel
  int* status;                // BM_ETIMEOUT when a barrier wait gave up
  int bar_sel;                // which counter this launch uses
};

struct GroupSmem {
  int cenT, stage, acc, cnt, live, lab, dtl, red, total;
};

__host__ __device__ inline GroupSmem group_smem(int npad_max, int kpad_max, int acc_floats) {
  GroupSmem L;
  int o = 0;
  L.cenT = o;  o += align_up(npad_max * (kpad_max + 1) * 4, 16);   // centroids [f][kpad + 1]
  L.stage = o; o += align_up(64 * npad_max * 4, 16);         // staged tile
  L.acc = o;   o += align_up(acc_floats * 4, 16);            // [ng][k][npad] sums
  L.cnt = o;   o += align_up(8 * kpad_max * 4, 16);          // [ng][k] counts
  L.live = o;  o += align_up(kpad_max * 4, 16);
  L.lab = o;   o += 64 * 4;
  L.dtl = o;   o += 64 * 4;                                  // row-lane shape: distances
  L.red = o;   o += 40 * 8;
  L.total = o;
  return L;
}

// Nearest live centroid of the 64 staged rows with four lanes per row (k <=
// 16): thread t takes row t / 4 and centroids t % 4, t % 4 + 4, ...; each
// distance is the sum over features in order of the squared differences,
// as in nearest_tile, and ties go to the lowest index.  The result reaches
// the thread that nearest_tile would give it (lane r of warp w for row
// 8w + r), through shared memory; same contract as nearest_tile.
__device__ __forceinline__ bool nearest_tile_rows(const float* stage, const float* cenT,
                                                  const int* live, int k, int cs, int n,
                                                  int rows, int* lab_s, float* d_s,
                                                  int& bj, float& bd) {
  const int t = threadIdx.x, r = t >> 2, sub = t & 3;
  const int nq = (k + 3) >> 2;   // centroids per lane (at most 4)
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int f = 0; f < n; ++f) {
    const float x = stage[f * 64 + (r ^ swz(f))];
    const float* cf = cenT + f * cs + sub;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq) acc[q] = sq(x - cf[4 * q], acc[q]);
  }
  float d = INFINITY;
  int j = INT_MAX;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = sub + 4 * q;
    if (q < nq && jj < k && live[jj] && (j == INT_MAX || acc[q] < d)) {
      d = acc[q];
      j = jj;
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    const float od = __shfl_xor_sync(0xffffffffu, d, o);
    const int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (better(od, oj, d, j)) { d = od; j = oj; }
  }
  if (sub == 0) { lab_s[r] = j; d_s[r] = d; }
  __syncthreads();
  const int w = t >> 5, l = t & 31;
  if (l < 8) {
    bj = lab_s[w * 8 + l];
    bd = d_s[w * 8 + l];
    return w * 8 + l < rows;
  }
  return false;
}

// The assignment phase: every segment of this CTA (see the file comment).
__device__ void group_assign_segments(const GroupArgs& a) {
  extern __shared__ __align__(16) char gsm[];
  const GroupSmem L = group_smem(a.npad_max, a.kpad_max, a.acc_floats);
  float* cenT = reinterpret_cast<float*>(gsm + L.cenT);
  float* stage = reinterpret_cast<float*>(gsm + L.stage);
  float* acc = reinterpret_cast<float*>(gsm + L.acc);
  int* cnt = reinterpret_cast<int*>(gsm + L.cnt);
  int* live = reinterpret_cast<int*>(gsm + L.live);
  int* lab = reinterpret_cast<int*>(gsm + L.lab);
  float* dtl = reinterpret_cast<float*>(gsm + L.dtl);
  double* red = reinterpret_cast<double*>(gsm + L.red);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int sg = a.cta_seg[blockIdx.x]; sg < a.cta_seg[blockIdx.x + 1]; ++sg) {
    const GroupSeg seg = a.segs[sg];
    if (__ldcg(&a.st[seg.prob].done)) continue;   // uniform over the CTA
    const GroupProb p = a.probs[seg.prob];
    const int n = p.n, npad = p.npad, k = p.k, kpad = p.kpad, ng = p.ng;
    // centroid rows are kpad + 1 floats apart, so that the update's reads of
    // one centroid's features fall in different banks (the scan reads rows)
    const int cs = kpad + 1;
    __syncthreads();   // the previous segment is done with shared memory
    for (int e = threadIdx.x; e < npad * kpad; e += blockDim.x) {
      const int f = e / kpad, j = e - f * kpad;
      cenT[f * cs + j] = (j < k && f < n) ? __ldcg(p.C + (size_t)j * n + f) : 0.f;
    }
    for (int j = threadIdx.x; j < kpad; j += blockDim.x)
      live[j] = j < k && __ldcg(reinterpret_cast<const unsigned char*>(p.mask) + j) != 0;
    for (int q = threadIdx.x; q < ng * k * npad; q += blockDim.x) acc[q] = 0.f;
    for (int q = threadIdx.x; q < ng * k; q += blockDim.x) cnt[q] = 0;
    __syncthreads();
    const bool vec4 = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.P) & 15) == 0);
    double fa = 0.0;
    for (int t = seg.t0; t < seg.t1; ++t) {
      const long long r0 = (long long)t * 64;
      const int rows = (int)min(64LL, p.s - r0);
      stage_tile(stage, p.P + (size_t)r0 * n, n, rows, n, npad, vec4, false);
      int j;
      float d;
      // (nearest_tile takes the row stride as its kpad: cs >> 5 == kpad >> 5)
      const bool mine = p.rows_tile ? nearest_tile_rows(stage, cenT, live, k, cs, n, rows, lab,
                                                        dtl, j, d)
                                    : nearest_tile(stage, cenT, live, k, cs, n, rows, j, d);
      __syncthreads();   // the row-lane shape's results are read before lab is rewritten
      if (mine) {
        const int r = w * 8 + l;
        lab[r] = j;
        fa += (double)d;
        if (p.labels) p.labels[r0 + r] = j;
      }
      __syncthreads();
      // thread (g, f) adds rows g, g + ng, ... of the tile in order
      for (int slot = threadIdx.x; slot < ng * npad; slot += blockDim.x) {
        const int g = slot / npad, f = slot - g * npad;
        if (f >= n) continue;
        float* ag = acc + (size_t)g * k * npad;
        const int sz = swz(f);
        for (int r = g; r < rows; r += ng) {
          const int jr = lab[r];
          if (jr >= k) continue;
          ag[jr * npad + f] += stage[f * 64 + (r ^ sz)] - cenT[f * cs + jr];
          if (f == 0) cnt[g * k + jr] += 1;
        }
      }
      __syncthreads();
    }
    // the segment's slot: groups added in order
    const GroupSlotOff off = a.offs[sg];
    for (int q = threadIdx.x; q < k * npad; q += blockDim.x) {
      float sum = 0.f;
      for (int g = 0; g < ng; ++g) sum += acc[(size_t)g * k * npad + q];
      a.part_sum[off.sum + q] = sum;
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      int c = 0;
      for (int g = 0; g < ng; ++g) c += cnt[g * k + j];
      a.part_cnt[off.cnt + j] = c;
    }
    const double tot = block_sum_f64(fa, red);
    if (threadIdx.x == 0) a.part_f[sg] = tot;
  }
}

__global__ void __launch_bounds__(kGroupThreads)
group_assign_kernel(GroupArgs a) {
  BM_POISON_SMEM();
  group_assign_segments(a);
}

// The update phase of problem pi (one CTA).
__device__ void group_update_one(const GroupArgs& a, int pi) {
  GroupState* st = a.st + pi;
  if (__ldcg(&st->done)) return;   // uniform over the CTA
  const GroupProb p = a.probs[pi];
  const int n = p.n, npad = p.npad, k = p.k;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __shared__ double s_f;
  __shared__ int s_live0, s_live1;
  if (w == 0) {
    double v = 0.0;
    for (int i = p.slot0 + l; i < p.slot1; i += 32) v += __ldcg(a.part_f + i);
    v = warp_sum_f64(v);
    int lv = 0;
    for (int j = l; j < k; j += 32) lv += __ldcg(reinterpret_cast<const unsigned char*>(p.mask) + j) != 0;
    lv = warp_sum_i32(lv);
    if (l == 0) { s_f = v; s_live0 = lv; }
  }
  __syncthreads();
  const double f = s_f;
  const int it = st->it;
  const bool stop = (f == 0.0) || (it > 0 && st->f_prev - f <= a.tol * st->f_prev) ||
                    (it == a.max_iter);
  for (int q = threadIdx.x; q < k * n; q += blockDim.x) {
    const int j = q / n, f0 = q - j * n;
    if (!p.mask[j]) continue;
    int c = 0;
    float sum = 0.f;
    for (int i = p.slot0; i < p.slot1; ++i) {
      const GroupSlotOff off = a.offs[i];
      c += __ldcg(a.part_cnt + off.cnt + j);
      sum += __ldcg(a.part_sum + off.sum + (size_t)j * npad + f0);
    }
    if (c == 0) continue;   // degenerate: marked below, once every thread has read the mask
    if (!stop) p.C[(size_t)j * n + f0] += sum / (float)c;
  }
  __syncthreads();
  // live centroids without members become degenerate (Sec. 3.3)
  if (w == 0) {
    int lv = 0;
    for (int j = l; j < k; j += 32) {
      if (!p.mask[j]) continue;
      int c = 0;
      for (int i = p.slot0; i < p.slot1; ++i) c += __ldcg(a.part_cnt + a.offs[i].cnt + j);
      if (c == 0) p.mask[j] = 0;
      else ++lv;
    }
    lv = warp_sum_i32(lv);
    if (l == 0) s_live1 = lv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->f = f;
    st->nd += p.s * (long long)s_live0;
    st->live = s_live1;
    if (stop) {
      st->done = 1;
      atomicSub(a.active, 1);
    } else {
      st->f_prev = f;
      st->it = it + 1;
    }
  }
  __syncthreads();   // the CTA's next problem reuses the shared scalars
}

__global__ void __launch_bounds__(kGroupThreads)
group_update_kernel(GroupArgs a) {
  group_update_one(a, blockIdx.x);
}

// One Lloyd step of every unfinished problem in one cooperative launch.
__global__ void __launch_bounds__(kGroupThreads)
group_step_kernel(GroupArgs a) {
  BM_POISON_SMEM();
  BM_START_SKEW();
  group_assign_segments(a);
  GridBarrier gb{a.bar + a.bar_sel, a.status, 0u};
  if (!gb.sync()) return;
  for (int pi = blockIdx.x; pi < a.count; pi += gridDim.x) group_update_one(a, pi);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.bar[a.bar_sel ^ 1] = 0u;   // ready for the next launch
}

__global__ void group_reset_kernel(GroupState* st, int count, int* active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) st[i] = GroupState{0.0, 0.0, 0, 0, 0, 0, 0};
  if (i == 0) *active = count;
}

}  // namespace bm

using namespace bm;

struct bm_group {
  int device = 0;
  cudaStream_t stream = nullptr;
  int count = 0, grid = 0, nseg = 0, max_seg = 0;
  bool coop = false;            // the grid is co-resident: one launch per step
  int tiles_mode = 0;           // 0: autotune, 1: lane per centroid, 2: lanes per row (k <= 16)
  bool tuned = false;           // the tile shapes are chosen
  int nseg_all = 0;             // segments of the partition of every problem
  bool balance = true;
  size_t smem = 0;
  int max_iter = 300;
  GroupArgs args{};
  void* dev_block = nullptr;    // every device array of the group, one allocation
  int* active_host = nullptr;   // pinned
  std::vector<GroupProb> hp;    // problems (host copy; slots rewritten per partition)
  std::vector<int> tiles;       // 64-row tiles per problem
  std::vector<double> tile_cost;
  long long sum_cap = 0, cnt_cap = 0;   // room of the partial-result arrays
  cudaGraphExec_t graph = nullptr;
};

namespace {

bm_status group_free(bm_group* g) {
  if (!g) return BM_OK;
  if (g->graph) cudaGraphExecDestroy(g->graph);
  if (g->dev_block) cudaFree(g->dev_block);
  if (g->active_host) cudaFreeHost(g->active_host);
  delete g;
  return BM_OK;
}

// One cooperative launch per Lloyd step (the grid barrier alternates
// between two counters: step i uses counter i % 2 and clears the other; the
// step count of a recorded graph is even), else an assignment and an update
// launch per step.
bm_status enqueue_steps(bm_group* g, int steps) {
  const int gu = g->count;
  for (int i = 0; i < steps; ++i) {
    if (g->coop) {
      GroupArgs a = g->args;
      a.bar_sel = i & 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(g->grid);
      cfg.blockDim = dim3(kGroupThreads);
      cfg.dynamicSmemBytes = g->smem;
      cfg.stream = g->stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, group_step_kernel, a) != cudaSuccess) return BM_ECUDA;
    } else {
      group_assign_kernel<<<g->grid, kGroupThreads, g->smem, g->stream>>>(g->args);
      group_update_kernel<<<gu, kGroupThreads, 0, g->stream>>>(g->args);
    }
  }
  return cudaGetLastError() == cudaSuccess ? BM_OK : BM_ECUDA;
}

// Cuts the tiles of the problems with active[i] set into per-CTA ranges of
// equal cost (balance) or gives each such problem one CTA, assigns the
// segments their slots, and uploads the tables on the group's stream.  Every
// problem's slots are adjacent and in CTA order.
bm_status group_partition(bm_group* g, const std::vector<char>& active) {
  const int count = g->count, grid = g->grid;
  std::vector<GroupSeg> segs;
  std::vector<int> cta_seg;
  if (g->balance) {
    double total = 0.0;
    for (int i = 0; i < count; ++i)
      if (active[i]) total += g->tile_cost[i] * g->tiles[i];
    const double per = total > 0.0 ? total / grid : 1.0;
    double acc = 0.0;
    int cta = 0;
    cta_seg.push_back(0);
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      for (int t = 0; t < g->tiles[i]; ++t) {
        // a tile goes to the CTA whose range holds its cost midpoint
        const int want = std::min(grid - 1, (int)((acc + 0.5 * g->tile_cost[i]) / per));
        while (cta < want) {
          ++cta;
          cta_seg.push_back((int)segs.size());
        }
        if (cta_seg.back() < (int)segs.size() && segs.back().prob == i && segs.back().t1 == t)
          segs.back().t1 = t + 1;
        else
          segs.push_back(GroupSeg{i, t, t + 1});
        acc += g->tile_cost[i];
      }
    }
    while (cta < grid - 1) {
      ++cta;
      cta_seg.push_back((int)segs.size());
    }
    cta_seg.push_back((int)segs.size());
  } else {
    // grid == count: CTA i owns problem i
    for (int i = 0; i < count; ++i) {
      cta_seg.push_back((int)segs.size());
      if (active[i]) segs.push_back(GroupSeg{i, 0, g->tiles[i]});
    }
    cta_seg.push_back((int)segs.size());
  }
  const int nseg = (int)segs.size();
  if (nseg > g->max_seg) return BM_ECUDA;   // cannot happen: nseg <= grid + count
  std::vector<GroupSlotOff> offs(nseg);
  long long sum_total = 0, cnt_total = 0;
  for (int i = 0; i < count; ++i) { g->hp[i].slot0 = 0; g->hp[i].slot1 = 0; }
  std::vector<char> seen(count, 0);
  for (int sg = 0; sg < nseg; ++sg) {
    GroupProb& p = g->hp[segs[sg].prob];
    offs[sg].sum = sum_total;
    offs[sg].cnt = cnt_total;
    sum_total += (long long)p.k * p.npad;
    cnt_total += p.k;
    if (!seen[segs[sg].prob]) { p.slot0 = sg; seen[segs[sg].prob] = 1; }
    p.slot1 = sg + 1;
  }
  if (sum_total > g->sum_cap || cnt_total > g->cnt_cap) return BM_ECUDA;
  g->nseg = nseg;
  cudaStream_t st = g->stream;
  GroupArgs& ga = g->args;
  if (cudaMemcpyAsync((void*)ga.probs, g->hp.data(), sizeof(GroupProb) * count,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (nseg > 0 && cudaMemcpyAsync((void*)ga.segs, segs.data(), sizeof(GroupSeg) * nseg,
                                   cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      (nseg > 0 && cudaMemcpyAsync((void*)ga.offs, offs.data(), sizeof(GroupSlotOff) * nseg,
                                   cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaMemcpyAsync((void*)ga.cta_seg, cta_seg.data(), sizeof(int) * cta_seg.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {   // the host vectors die here
    cudaGetLastError();
    return BM_ECUDA;
  }
  return BM_OK;
}

// Tile shapes (see the file comment).  Mode 1 keeps a lane per centroid, mode
// 2 takes four lanes per row wherever k <= 16; mode 0 times both on the
// problems of each (n, k) with k <= 16 -- one assignment launch each after a
// warm-up, CUDA events on the group's stream -- and keeps the faster.  The
// shapes give the same bits, so the choice only changes the time.
bm_status group_tune(bm_group* g) {
  const int count = g->count;
  std::map<std::pair<int, int>, std::vector<int>> shapes;
  for (int i = 0; i < count; ++i) {
    GroupProb& p = g->hp[i];
    p.rows_tile = (g->tiles_mode == 2 && p.k <= 16) ? 1 : 0;
    if (g->tiles_mode == 0 && p.k <= 16) shapes[{p.n, p.k}].push_back(i);
  }
  if (shapes.empty()) return BM_OK;
  cudaStream_t st = g->stream;
  group_reset_kernel<<<(count + 255) / 256, 256, 0, st>>>(g->args.st, count, g->args.active);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaGetLastError() != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return BM_ECUDA;
  }
  bm_status rc = BM_OK;
  for (auto& kv : shapes) {
    std::vector<char> act(count, 0);
    for (int i : kv.second) act[i] = 1;
    float ms[2] = {0.f, 0.f};
    for (int shape = 0; shape < 2 && rc == BM_OK; ++shape) {
      for (int i : kv.second) g->hp[i].rows_tile = shape;
      rc = group_partition(g, act);
      if (rc != BM_OK) break;
      group_assign_kernel<<<g->grid, kGroupThreads, g->smem, st>>>(g->args);   // warm-up
      cudaEventRecord(e0, st);
      group_assign_kernel<<<g->grid, kGroupThreads, g->smem, st>>>(g->args);
      cudaEventRecord(e1, st);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms[shape], e0, e1) != cudaSuccess)
        rc = BM_ECUDA;
    }
    const int pick = ms[1] < ms[0] ? 1 : 0;
    for (int i : kv.second) g->hp[i].rows_tile = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != BM_OK) cudaGetLastError();
  return rc;
}

}  // namespace

extern "C" {

bm_status bm_group_set_tiles(bm_group* g, int32_t mode) {
  if (!g || mode < 0 || mode > 2) return BM_EINVAL;
  g->tiles_mode = mode;
  g->tuned = false;
  return BM_OK;
}

bm_status bm_group_tiles(bm_group* g, int32_t* shapes_host) {
  if (!g || !shapes_host) return BM_EINVAL;
  for (int i = 0; i < g->count; ++i) shapes_host[i] = g->hp[i].rows_tile;
  return BM_OK;
}

bm_status bm_group_create(const bm_group_problem* probs, int32_t count, int32_t max_iter,
                          double tol, int32_t balance, void* stream, bm_group** out) {
  if (!out) return BM_EINVAL;
  *out = nullptr;
  if (!probs || count < 1 || max_iter < 0 || !(tol >= 0.0)) return BM_EINVAL;
  int npad_max = 4, kpad_max = 32, kn_max = 1;
  for (int i = 0; i < count; ++i) {
    const bm_group_problem& q = probs[i];
    if (!q.P_dev || !q.C_dev || !q.mask_dev || q.s < 1 || q.n < 1 || q.k < 1 || q.k > q.s)
      return BM_EINVAL;
    if (q.k > 128 || q.n > 512 || (q.s + 63) / 64 > INT_MAX) return BM_EUNSUPPORTED;
    const int npad = align_up(q.n, 4), kpad = align_up(q.k, 32);
    npad_max = std::max(npad_max, npad);
    kpad_max = std::max(kpad_max, kpad);
    kn_max = std::max(kn_max, q.k * npad);
  }
  // accumulators: room for one [k][npad] copy of the widest problem, at
  // least 16 KB; narrower problems use the room for more row groups
  const int acc_floats = std::max(kn_max, 4096);
  const GroupSmem L = group_smem(npad_max, kpad_max, acc_floats);
  if ((size_t)L.total > kGroupSmemLimit) return BM_EUNSUPPORTED;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return BM_ECUDA; }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (allow_max_smem(group_assign_kernel) != cudaSuccess ||
      allow_max_smem(group_step_kernel) != cudaSuccess)
    return BM_ECUDA;
  int per_sm = 0, per_sm_step = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, group_assign_kernel,
                                                    kGroupThreads, L.total) != cudaSuccess ||
      per_sm < 1 ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_step, group_step_kernel,
                                                    kGroupThreads, L.total) != cudaSuccess)
    return BM_EUNSUPPORTED;
  per_sm = std::min(per_sm, std::max(per_sm_step, 1));

  bm_group* g = new (std::nothrow) bm_group();
  if (!g) return BM_ENOMEM;
  g->device = dev;
  g->stream = static_cast<cudaStream_t>(stream);
  g->count = count;
  g->balance = balance != 0;
  g->grid = g->balance ? per_sm * sms : count;
  g->coop = per_sm_step >= 1 && g->grid <= per_sm_step * sms;
  g->smem = L.total;
  g->max_iter = max_iter;
  g->hp.resize(count);
  g->tiles.resize(count);
  g->tile_cost.resize(count);
  for (int i = 0; i < count; ++i) {
    const bm_group_problem& q = probs[i];
    GroupProb& p = g->hp[i];
    p.P = q.P_dev;
    p.C = q.C_dev;
    p.mask = q.mask_dev;
    p.labels = q.labels_dev;
    p.s = q.s;
    p.n = q.n;
    p.npad = align_up(q.n, 4);
    p.k = q.k;
    p.kpad = align_up(q.k, 32);
    int ng = std::min(kGroupThreads / p.npad, acc_floats / (p.k * p.npad));
    p.ng = std::max(1, std::min(ng, 8));
    p.rows_tile = 0;
    g->tiles[i] = (int)((q.s + 63) / 64);
    g->tile_cost[i] = (double)q.n * (double)(p.kpad / 32 + 1);
  }
  // any partition has at most grid + count segments; each slot holds one
  // problem's [k][npad] sums and [k] counts
  g->max_seg = g->grid + count;
  long long kn_big = 0, k_big = 0;
  for (int i = 0; i < count; ++i) {
    kn_big = std::max(kn_big, (long long)g->hp[i].k * g->hp[i].npad);
    k_big = std::max(k_big, (long long)g->hp[i].k);
  }
  g->sum_cap = kn_big * g->max_seg;
  g->cnt_cap = k_big * g->max_seg;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t b_probs = al(sizeof(GroupProb) * count);
  const size_t b_segs = al(sizeof(GroupSeg) * g->max_seg);
  const size_t b_offs = al(sizeof(GroupSlotOff) * g->max_seg);
  const size_t b_cta = al(sizeof(int) * (g->grid + 1));
  const size_t b_sum = al(sizeof(float) * (size_t)g->sum_cap);
  const size_t b_cnt = al(sizeof(int) * (size_t)g->cnt_cap);
  const size_t b_f = al(sizeof(double) * g->max_seg);
  const size_t b_st = al(sizeof(GroupState) * count);
  const size_t b_act = al(sizeof(int));
  const size_t b_ctl = al(4 * sizeof(int));   // barrier counters [2], status
  const size_t bytes = b_probs + b_segs + b_offs + b_cta + b_sum + b_cnt + b_f + b_st + b_act +
                       b_ctl;
  if (cudaMalloc(&g->dev_block, bytes) != cudaSuccess ||
      cudaMallocHost(&g->active_host, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    group_free(g);
    return BM_ENOMEM;
  }
  char* base = static_cast<char*>(g->dev_block);
  GroupArgs& ga = g->args;
  size_t o = 0;
  ga.probs = reinterpret_cast<GroupProb*>(base + o); o += b_probs;
  ga.segs = reinterpret_cast<GroupSeg*>(base + o); o += b_segs;
  ga.offs = reinterpret_cast<GroupSlotOff*>(base + o); o += b_offs;
  ga.cta_seg = reinterpret_cast<int*>(base + o); o += b_cta;
  ga.part_sum = reinterpret_cast<float*>(base + o); o += b_sum;
  ga.part_cnt = reinterpret_cast<int*>(base + o); o += b_cnt;
  ga.part_f = reinterpret_cast<double*>(base + o); o += b_f;
  ga.st = reinterpret_cast<GroupState*>(base + o); o += b_st;
  ga.active = reinterpret_cast<int*>(base + o); o += b_act;
  ga.bar = reinterpret_cast<uint32_t*>(base + o);
  ga.status = reinterpret_cast<int*>(base + o + 2 * sizeof(uint32_t));
  if (cudaMemset(ga.bar, 0, b_ctl) != cudaSuccess) {
    cudaGetLastError();
    group_free(g);
    return BM_ECUDA;
  }
  ga.count = count;
  ga.max_iter = max_iter;
  ga.tol = tol;
  ga.npad_max = npad_max;
  ga.kpad_max = kpad_max;
  ga.acc_floats = acc_floats;
  const bm_status rc = group_partition(g, std::vector<char>(count, 1));
  if (rc != BM_OK) {
    group_free(g);
    return rc;
  }
  g->nseg_all = g->nseg;
  *out = g;
  return BM_OK;
}

bm_status bm_group_run(bm_group* g, bm_group_result* results, int32_t* steps_out) {
  if (!g) return BM_EINVAL;
  cudaStream_t st = g->stream;
  if (!g->tuned) {
    const bm_status trc = group_tune(g);
    if (trc != BM_OK) return trc;
    g->tuned = true;
  }
  std::vector<char> active(g->count, 1);
  bm_status rc = group_partition(g, active);
  if (rc != BM_OK) return rc;
  group_reset_kernel<<<(g->count + 255) / 256, 256, 0, st>>>(g->args.st, g->count, g->args.active);
  if (cudaGetLastError() != cudaSuccess) return BM_ECUDA;
  if (!g->graph && st != nullptr) {
    // record a few steps once; replays re-read every table from device memory
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return BM_ECUDA;
    }
    const bm_status erc = enqueue_steps(g, kGroupStepsPerGraph);
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (erc != BM_OK || ce != cudaSuccess ||
        cudaGraphInstantiate(&g->graph, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      g->graph = nullptr;
      cudaGetLastError();
      return BM_ECUDA;
    }
    cudaGraphDestroy(graph);
  }
  // every problem stops within max_iter + 1 assignments
  const int max_steps = g->max_iter + 1;
  std::vector<GroupState> hs(g->count);
  int steps = 0, last_active = g->count;
  while (true) {
    if (g->graph) {
      if (cudaGraphLaunch(g->graph, st) != cudaSuccess) { cudaGetLastError(); return BM_ECUDA; }
    } else if (enqueue_steps(g, kGroupStepsPerGraph) != BM_OK) {   // legacy stream: no capture
      return BM_ECUDA;
    }
    steps += kGroupStepsPerGraph;
    if (cudaMemcpyAsync(g->active_host, g->args.active, sizeof(int), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return BM_ECUDA;
    }
    const int now = *g->active_host;
    int status = 0;
    if (g->coop && cudaMemcpy(&status, g->args.status, sizeof(int), cudaMemcpyDeviceToHost) !=
                       cudaSuccess) {
      cudaGetLastError();
      return BM_ECUDA;
    }
    if (status != 0) {   // a barrier wait gave up: clear the counters for the next run
      cudaMemset(g->args.bar, 0, 4 * sizeof(int));
      cudaDeviceSynchronize();
      return (bm_status)status;
    }
    if (now <= 0) break;
    if (steps >= max_steps + kGroupStepsPerGraph) return BM_ECUDA;   // cannot happen
    if (now < last_active && g->balance) {
      // spread the unfinished problems over the whole GPU again
      if (cudaMemcpy(hs.data(), g->args.st, sizeof(GroupState) * g->count,
                     cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return BM_ECUDA;
      }
      for (int i = 0; i < g->count; ++i) active[i] = hs[i].done == 0;
      rc = group_partition(g, active);
      if (rc != BM_OK) return rc;
      last_active = now;
    }
  }
  if (results) {
    if (cudaMemcpyAsync(hs.data(), g->args.st, sizeof(GroupState) * g->count,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return BM_ECUDA;
    }
    for (int i = 0; i < g->count; ++i) {
      results[i].f = hs[i].f;
      results[i].iters = hs[i].it;
      results[i].live = hs[i].live;
      results[i].n_d = hs[i].nd;
    }
  }
  if (steps_out) *steps_out = steps;
  return BM_OK;
}

bm_status bm_group_info(bm_group* g, int32_t* grid_out, int32_t* segments_out,
                        int64_t* smem_out) {
  if (!g) return BM_EINVAL;
  if (grid_out) *grid_out = g->grid;
  if (segments_out) *segments_out = g->nseg_all;
  if (smem_out) *smem_out = (int64_t)g->smem;
  return BM_OK;
}

bm_status bm_group_destroy(bm_group* g) {
  if (g && g->stream) cudaStreamSynchronize(g->stream);
  return group_free(g);
}

}  // extern "C"
