// Grouped Lloyd: many independent Lloyd problems (Sec. 2, stop rule of
// Sec. 5) advanced together, one pair of launches per Lloyd step for all of
// them (bm_group_create / bm_group_run / bm_group_destroy).
//
// Work layout.  Every problem's rows form 64-row tiles; the tiles of all
// problems, problem after problem, form one list, and the list is cut into
// one contiguous range per CTA of equal estimated cost (a tile of problem p
// costs about n_p * (ceil(k_p / 32) + 1)), so a large problem spreads over
// many SMs and small ones share an SM.  The part of a CTA's range that lies
// in one problem is a segment; a segment owns a slot of partial results.
//
//   group_assign_kernel  (grid: the CTAs of the partition)
//     per segment of an unfinished problem: the problem's centroids into
//     shared memory, then per tile the nearest live centroid of each row
//     (the tiled FP32 arithmetic of the chunk kernels, lowest index on
//     ties), the row's label, and the row's (x - c_label) added into
//     per-row-group accumulators in a fixed row order; at the end the
//     segment's sums, member counts and objective go to its slot.
//   group_update_kernel  (grid: one CTA per problem)
//     per unfinished problem: its slots added in CTA order (the objective in
//     float64), the stop test, degenerate marking of live centroids without
//     members, the centroid update unless stopping, and the problem's state.
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
#include <new>
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
};

struct GroupSmem {
  int cenT, stage, acc, cnt, live, lab, red, total;
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
  L.red = o;   o += 40 * 8;
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(kGroupThreads)
group_assign_kernel(GroupArgs a) {
  extern __shared__ __align__(16) char gsm[];
  const GroupSmem L = group_smem(a.npad_max, a.kpad_max, a.acc_floats);
  float* cenT = reinterpret_cast<float*>(gsm + L.cenT);
  float* stage = reinterpret_cast<float*>(gsm + L.stage);
  float* acc = reinterpret_cast<float*>(gsm + L.acc);
  int* cnt = reinterpret_cast<int*>(gsm + L.cnt);
  int* live = reinterpret_cast<int*>(gsm + L.live);
  int* lab = reinterpret_cast<int*>(gsm + L.lab);
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
      if (nearest_tile(stage, cenT, live, k, cs, n, rows, j, d)) {
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
group_update_kernel(GroupArgs a) {
  const int pi = blockIdx.x;
  GroupState* st = a.st + pi;
  if (__ldcg(&st->done)) return;
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

bm_status enqueue_steps(bm_group* g, int steps) {
  const int gu = g->count;
  for (int i = 0; i < steps; ++i) {
    group_assign_kernel<<<g->grid, kGroupThreads, g->smem, g->stream>>>(g->args);
    group_update_kernel<<<gu, kGroupThreads, 0, g->stream>>>(g->args);
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

}  // namespace

extern "C" {

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
  if (allow_max_smem(group_assign_kernel) != cudaSuccess) return BM_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, group_assign_kernel,
                                                    kGroupThreads, L.total) != cudaSuccess ||
      per_sm < 1)
    return BM_EUNSUPPORTED;

  bm_group* g = new (std::nothrow) bm_group();
  if (!g) return BM_ENOMEM;
  g->device = dev;
  g->stream = static_cast<cudaStream_t>(stream);
  g->count = count;
  g->balance = balance != 0;
  g->grid = g->balance ? per_sm * sms : count;
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
  const size_t bytes = b_probs + b_segs + b_offs + b_cta + b_sum + b_cnt + b_f + b_st + b_act;
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
  ga.active = reinterpret_cast<int*>(base + o);
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
