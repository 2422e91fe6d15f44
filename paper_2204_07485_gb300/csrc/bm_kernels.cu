// Big-means hot path on sm_103a.
//
// chunk_kernel: one cooperative launch per chunk runs Alg. 1's loop body on
// the whole GPU -- sample draw (Sec. 3.5), gather P = X[idx], K-means++ reseed
// of degenerate centroids (Sec. 3.3, three candidates per Sec. 5), Lloyd
// iterations (Sec. 2) with the stop rule of Sec. 5, and keep-the-best
// (Alg. 1) -- separated by bounded-wait grid barriers instead of kernel
// launches.  Every CTA owns a fixed block of R = ceil(s / G) sample rows;
// every cross-CTA reduction has a fixed shape and order, so results are
// bitwise reproducible for a given grid.
//
// assign kernels: the final assignment of Alg. 1 (Sec. 3.4), streaming X once
// from HBM with a float64 sum of the per-row minima.
//
// Distances are evaluated as sum_f (x_f - c_f)^2 in FP32 (direct difference,
// not the ||x||^2 - 2 x.c + ||c||^2 expansion, which loses digits when the
// norms are large against the distance).  Two layouts:
//   - n <= 32 ("np" path): one thread per row with the row in registers, the
//     centroid table row-major in shared memory read as broadcast float4;
//   - n > 32 ("generic" path): 64-row tiles staged transposed in shared
//     memory; each warp takes 8 rows and each lane one centroid per group of
//     32, centroids transposed [f][kpad] in shared memory; the per-row argmin
//     is a fixed-order warp shuffle (lowest index on ties).
#include <cfloat>
#include <climits>

#include "bm_device.cuh"
#include "bm_internal.h"

namespace bm {

// ---------------------------------------------------------------- smem view
struct Smem {
  float* cen;   // np: [k][npad]   generic: [npad][kpad]
  int* live;    // [k]
  float* sw;    // [wu][k][32] per-warp update slices
  int* cw;      // [wu][k] per-warp member counts
  int* lab;     // [R] labels of own rows
  float* dmin;  // [R] nearest squared distance / K-means++ D^2 of own rows
  float* dc;    // [kMaxTrials][R] candidate distances of own rows
  float* cand;  // [kMaxTrials][npad] candidate rows
  float* stage; // [npad][64] transposed row tile (generic)
  double* red;  // scratch for block reductions (64 doubles)
};

__device__ __forceinline__ Smem carve(char* base, const ChunkSmem& L) {
  Smem S;
  S.cen = reinterpret_cast<float*>(base + L.cen);
  S.live = reinterpret_cast<int*>(base + L.live);
  S.sw = reinterpret_cast<float*>(base + L.sw);
  S.cw = reinterpret_cast<int*>(base + L.cw);
  S.lab = reinterpret_cast<int*>(base + L.lab);
  S.dmin = reinterpret_cast<float*>(base + L.dmin);
  S.dc = reinterpret_cast<float*>(base + L.dc);
  S.cand = reinterpret_cast<float*>(base + L.cand);
  S.stage = reinterpret_cast<float*>(base + L.stage);
  S.red = reinterpret_cast<double*>(base + L.red);
  return S;
}

__device__ __forceinline__ float sq(float e, float acc) { return fmaf(e, e, acc); }

// Centroid row j (global, k x cstride) -> shared table, both layouts.
template <bool GENERIC>
__device__ void load_centroids(float* cen, int* live, const float* C,
                               int cstride, const uint8_t* mask, int k, int n,
                               int npad, int kpad, bool coherent) {
  for (int q = threadIdx.x; q < k * npad; q += kThreads) {
    const int j = q / npad, f = q - j * npad;
    float v = 0.f;
    if (f < n) v = coherent ? __ldcg(C + (size_t)j * cstride + f)
                            : __ldg(C + (size_t)j * cstride + f);
    if (GENERIC) cen[f * kpad + j] = v;
    else cen[j * npad + f] = v;
  }
  for (int j = threadIdx.x; j < k; j += kThreads) {
    const unsigned char mv = coherent
        ? __ldcg(reinterpret_cast<const unsigned char*>(mask) + j)
        : __ldg(reinterpret_cast<const unsigned char*>(mask) + j);
    live[j] = mv != 0;
  }
  __syncthreads();
}

// ------------------------------------------------------------ np path rows
template <int NP>
__device__ __forceinline__ void load_row_np(float (&p)[NP], const float* row,
                                            int n, bool vec4, bool coherent) {
  if (vec4) {
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4 * q < n)
        v = coherent ? __ldcg(reinterpret_cast<const float4*>(row) + q)
                     : __ldg(reinterpret_cast<const float4*>(row) + q);
      p[4 * q] = v.x; p[4 * q + 1] = v.y; p[4 * q + 2] = v.z; p[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int f = 0; f < NP; ++f)
      p[f] = f < n ? (coherent ? __ldcg(row + f) : __ldg(row + f)) : 0.f;
  }
}

template <int NP>
__device__ __forceinline__ void nearest_np(const float (&p)[NP],
                                           const float* cen, const int* live,
                                           int k, int& bj, float& bd) {
  bd = INFINITY;
  bj = INT_MAX;   // stays out of range when no centroid is live
  bool any = false;
  for (int j = 0; j < k; ++j) {
    if (!live[j]) continue;
    const float4* c4 = reinterpret_cast<const float4*>(cen + j * NP);
    float d = 0.f;
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
      const float4 c = c4[q];
      d = sq(p[4 * q] - c.x, d);
      d = sq(p[4 * q + 1] - c.y, d);
      d = sq(p[4 * q + 2] - c.z, d);
      d = sq(p[4 * q + 3] - c.w, d);
    }
    if (!any || d < bd) { bd = d; bj = j; any = true; }
  }
}

// -------------------------------------------------------- generic path rows
// stage[f][r] <- src[r][f] for r < rows (64-row tile), zero elsewhere.
__device__ void stage_tile(float* stage, const float* src, size_t stride,
                           int rows, int n, int npad, bool vec4, bool coherent) {
  if (vec4) {
    const int nq = npad / 4;
    for (int e = threadIdx.x; e < 64 * nq; e += kThreads) {
      const int r = e & 63, q = e >> 6;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows && 4 * q < n) {
        const float4* p = reinterpret_cast<const float4*>(src + (size_t)r * stride) + q;
        v = coherent ? __ldcg(p) : __ldg(p);
      }
      stage[(4 * q) * 64 + r] = v.x;
      stage[(4 * q + 1) * 64 + r] = v.y;
      stage[(4 * q + 2) * 64 + r] = v.z;
      stage[(4 * q + 3) * 64 + r] = v.w;
    }
  } else {
    for (int e = threadIdx.x; e < 64 * npad; e += kThreads) {
      const int r = e & 63, f = e >> 6;
      float v = 0.f;
      if (r < rows && f < n) {
        const float* p = src + (size_t)r * stride + f;
        v = coherent ? __ldcg(p) : __ldg(p);
      }
      stage[f * 64 + r] = v;
    }
  }
  __syncthreads();
}

// Nearest live centroid of the 64 staged rows; lane r of warp w reports tile
// row 8w + r through (bj, bd) and returns true when that row exists.
__device__ __forceinline__ bool nearest_tile(const float* stage,
                                             const float* cenT,
                                             const int* live, int k, int kpad,
                                             int n, int rows, int& bj,
                                             float& bd) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int kg = kpad >> 5;
  float acc[4][8];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[g][r] = 0.f;
  const float* sp = stage + w * 8;
  for (int f = 0; f < n; ++f) {
    const float4 pa = *reinterpret_cast<const float4*>(sp + f * 64);
    const float4 pb = *reinterpret_cast<const float4*>(sp + f * 64 + 4);
    const float* cf = cenT + f * kpad + l;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g < kg) {
        const float c = cf[g * 32];
        acc[g][0] = sq(pa.x - c, acc[g][0]);
        acc[g][1] = sq(pa.y - c, acc[g][1]);
        acc[g][2] = sq(pa.z - c, acc[g][2]);
        acc[g][3] = sq(pa.w - c, acc[g][3]);
        acc[g][4] = sq(pb.x - c, acc[g][4]);
        acc[g][5] = sq(pb.y - c, acc[g][5]);
        acc[g][6] = sq(pb.z - c, acc[g][6]);
        acc[g][7] = sq(pb.w - c, acc[g][7]);
      }
    }
  }
  bool mine = false;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float d = INFINITY;
    int j = INT_MAX;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int jj = g * 32 + l;
      if (g < kg && jj < k && live[jj] && (j == INT_MAX || acc[g][r] < d)) {
        d = acc[g][r];
        j = jj;
      }
    }
    warp_argmin(d, j);
    if (l == r) { bd = d; bj = j; mine = (w * 8 + r) < rows; }
  }
  return mine;
}

// ------------------------------------------------------ own-row assignment
// Nearest live centroid of every own row -> S.lab / S.dmin.
template <int NP, bool GENERIC>
__device__ void assign_own_rows(const ChunkArgs& a, const Smem& S, int r0,
                                int nrows) {
  if constexpr (!GENERIC) {
    for (int i = threadIdx.x; i < nrows; i += kThreads) {
      float p[NP];
      load_row_np<NP>(p, a.P + (size_t)(r0 + i) * a.npad, a.n, true, true);
      int j;
      float d;
      nearest_np<NP>(p, S.cen, S.live, a.k, j, d);
      S.lab[i] = j;
      S.dmin[i] = d;
    }
    __syncthreads();
  } else {
    for (int t0 = 0; t0 < nrows; t0 += 64) {
      const int rows = min(64, nrows - t0);
      stage_tile(S.stage, a.P + (size_t)(r0 + t0) * a.npad, a.npad, rows, a.n,
                 a.npad, true, true);
      int j;
      float d;
      if (nearest_tile(S.stage, S.cen, S.live, a.k, a.kpad, a.n, rows, j, d)) {
        const int i = t0 + (threadIdx.x >> 5) * 8 + (threadIdx.x & 31);
        S.lab[i] = j;
        S.dmin[i] = d;
      }
      __syncthreads();
    }
  }
}

// Fixed-order float64 sum of S.dmin over own rows (every thread gets it).
__device__ __forceinline__ double own_dmin_sum(const Smem& S, int nrows) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nrows; i += kThreads) v += (double)S.dmin[i];
  return block_sum_f64(v, S.red);
}

// Squared distances of own rows to the nc candidate rows in S.cand
// (warp per row, lanes over features) -> S.dc[c][i].
__device__ void own_rows_to_cands(const ChunkArgs& a, const Smem& S, int r0,
                                  int nrows, int nc) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int R = a.rows_per_cta;
  for (int i = w; i < nrows; i += kWarps) {
    float d[kMaxTrials];
#pragma unroll
    for (int c = 0; c < kMaxTrials; ++c) d[c] = 0.f;
    const float* row = a.P + (size_t)(r0 + i) * a.npad;
    for (int f = l; f < a.n; f += 32) {
      const float p = __ldcg(row + f);
#pragma unroll
      for (int c = 0; c < kMaxTrials; ++c)
        if (c < nc) d[c] = sq(p - S.cand[c * a.npad + f], d[c]);
    }
#pragma unroll
    for (int c = 0; c < kMaxTrials; ++c)
      if (c < nc) {
        const float t = warp_sum_f32(d[c]);
        if (l == 0) S.dc[c * R + i] = t;
      }
  }
  __syncthreads();
}

// Per-warp slices of sum_i (p_i - c_{label_i}) and member counts of own rows,
// combined over warps in a fixed order into part_sum[j][f][b], part_cnt[j][b].
template <bool GENERIC>
__device__ void update_partials(const ChunkArgs& a, const Smem& S,
                                const ChunkSmem& L, int r0, int nrows, int G) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int k = a.k, n = a.n, npad = a.npad, b = blockIdx.x;
  for (int fs = 0; fs < n; fs += 32) {
    if (w < L.wu) {
      float* my = S.sw + w * k * 32;
      for (int q = l; q < k * 32; q += 32) my[q] = 0.f;
      if (fs == 0)
        for (int j = l; j < k; j += 32) S.cw[w * k + j] = 0;
      __syncwarp();
      const int f = fs + l;
      for (int i = w; i < nrows; i += L.wu) {
        const int j = S.lab[i];
        if (j >= k) continue;   // no live centroid: nothing to accumulate
        if (f < n) {
          const float c = GENERIC ? __ldcg(a.C + (size_t)j * npad + f)
                                  : S.cen[j * npad + f];
          my[j * 32 + l] += __ldcg(a.P + (size_t)(r0 + i) * npad + f) - c;
        }
        if (fs == 0 && l == 0) S.cw[w * k + j] += 1;
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < k * 32; q += kThreads) {
      const int j = q >> 5, f = fs + (q & 31);
      if (f < n) {
        float sum = 0.f;
        for (int u = 0; u < L.wu; ++u) sum += S.sw[u * k * 32 + q];
        a.part_sum[((size_t)j * npad + f) * G + b] = sum;
      }
    }
    if (fs == 0)
      for (int j = threadIdx.x; j < k; j += kThreads) {
        int c = 0;
        for (int u = 0; u < L.wu; ++u) c += S.cw[u * k + j];
        a.part_cnt[(size_t)j * G + b] = c;
      }
    __syncthreads();
  }
}

// Block-wide exclusive scan of ints; *total receives the block sum.
__device__ __forceinline__ int block_excl_scan(int v, int* buf, int* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) buf[w] = x;
  __syncthreads();
  int before = 0, all = 0;
  for (int i = 0; i < kWarps; ++i) {
    if (i < w) before += buf[i];
    all += buf[i];
  }
  *total = all;
  return before + x - v;
}

// ------------------------------------------------------------------ phases
__device__ __forceinline__ uint32_t sample_word(const ChunkArgs& a, long long w,
                                                bool complement) {
  const uint32_t raw = __ldcg(a.bitmap + w);
  if (!complement) return raw;
  uint32_t v = ~raw;
  const long long lo = w * 32;
  if (lo + 32 > a.m) v &= (a.m - lo >= 32) ? 0xffffffffu : ((1u << (a.m - lo)) - 1u);
  return v;
}

// Sample draw: rounds of Philox draws deduplicated in the bitmap, then a
// fixed-order compaction of the set (or unset) bits into sorted indices.
__device__ bool phase_draw(const ChunkArgs& a, const Smem& S, GridBarrier& gb) {
  const bool complement = 2 * (long long)a.s > a.m;
  const uint32_t target = complement ? (uint32_t)(a.m - a.s) : (uint32_t)a.s;
  int* ired = reinterpret_cast<int*>(S.red);
  const unsigned long long gtid = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
  const unsigned long long gstride = (unsigned long long)gridDim.x * kThreads;
  uint32_t have = 0;
  if (target > 0) {
    for (int r = 0; r < kRoundSlots; ++r) {
      const uint32_t need = target - have;
      if (need == 0) break;
      int mine = 0;
      for (unsigned long long i = gtid; i < need; i += gstride) {
        const uint64_t w = philox_word(a.seed, (uint64_t)a.t, 0, (uint64_t)r, i);
        const uint64_t v = __umul64hi(w, (uint64_t)a.m);
        const uint32_t bit = 1u << (v & 31);
        const uint32_t old = atomicOr(a.bitmap + (v >> 5), bit);
        mine += (old & bit) ? 0 : 1;
      }
      const int blk = block_sum_i32(mine, ired);
      if (threadIdx.x == 0 && blk) atomicAdd(&a.ctl->round_cnt[r], (uint32_t)blk);
      if (!gb.sync()) return false;
      have += __ldcg(&a.ctl->round_cnt[r]);
    }
    if (have < target) {
      // Rounds exhausted (never in practice): the smallest absent values
      // complete the set.
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long W = (a.m + 31) / 32;
        for (long long w = 0; w < W && have < target; ++w) {
          uint32_t word = a.bitmap[w];
          for (int bpos = 0; bpos < 32 && have < target; ++bpos) {
            if (w * 32 + bpos >= a.m) break;
            if (!(word & (1u << bpos))) { word |= 1u << bpos; ++have; }
          }
          a.bitmap[w] = word;
        }
      }
      if (!gb.sync()) return false;
    }
  }
  // compaction: CTA b owns words [w0, w1)
  const long long W = (a.m + 31) / 32;
  const long long wb = (W + gridDim.x - 1) / gridDim.x;
  const long long w0 = min(W, (long long)blockIdx.x * wb), w1 = min(W, w0 + wb);
  int cnt = 0;
  for (long long w = w0 + threadIdx.x; w < w1; w += kThreads)
    cnt += __popc(sample_word(a, w, complement));
  cnt = block_sum_i32(cnt, ired);
  if (threadIdx.x == 0) a.blk_cnt[blockIdx.x] = cnt;
  if (!gb.sync()) return false;
  int base = 0;
  for (int q = threadIdx.x; q < (int)blockIdx.x; q += kThreads) base += __ldcg(a.blk_cnt + q);
  base = block_sum_i32(base, ired);
  for (long long t0 = w0; t0 < w1; t0 += kThreads) {
    const long long w = t0 + threadIdx.x;
    uint32_t bits = w < w1 ? sample_word(a, w, complement) : 0u;
    int tile_total;
    int pos = base + block_excl_scan(__popc(bits), ired + 16, &tile_total);
    while (bits) {
      const int bp = __ffs(bits) - 1;
      if (pos < a.s) a.idx[pos] = (int32_t)(w * 32 + bp);   // bound: stray bits
      ++pos;
      bits &= bits - 1;
    }
    base += tile_total;
  }
  __syncthreads();
  for (long long w = w0 + threadIdx.x; w < w1; w += kThreads) a.bitmap[w] = 0u;
  if (!gb.sync()) return false;
  if (blockIdx.x == 0)
    for (int r = threadIdx.x; r < kRoundSlots; r += kThreads) a.ctl->round_cnt[r] = 0u;
  return true;
}

// P[i] = X[idx[i]] for own rows (zero padding to npad).
__device__ void phase_gather(const ChunkArgs& a, int r0, int nrows) {
  const int npad = a.npad, n = a.n;
  for (int e = threadIdx.x; e < nrows * npad; e += kThreads) {
    const int i = e / npad, f = e - i * npad;
    float v = 0.f;
    if (f < n) {
      const long long row = __ldcg(a.idx + r0 + i);
      v = __ldg(a.X + (size_t)row * n + f);
    }
    a.P[(size_t)(r0 + i) * npad + f] = v;
  }
}

template <bool GENERIC>
__device__ __forceinline__ void set_centroid_row(const Smem& S, const float* src,
                                                 int j, int npad, int kpad) {
  for (int f = threadIdx.x; f < npad; f += kThreads) {
    if (GENERIC) S.cen[f * kpad + j] = src[f];
    else S.cen[j * npad + f] = src[f];
  }
}

__device__ __forceinline__ void load_cand_row(const ChunkArgs& a, const Smem& S,
                                              int c, int row) {
  for (int f = threadIdx.x; f < a.npad; f += kThreads)
    S.cand[c * a.npad + f] = __ldcg(a.P + (size_t)row * a.npad + f);
}

// K-means++ reseed of every degenerate slot, ascending (Sec. 3.3, Sec. 5).
template <int NP, bool GENERIC>
__device__ bool phase_kpp(const ChunkArgs& a, const Smem& S, GridBarrier& gb,
                          int r0, int nrows, long long* nd_out) {
  const int k = a.k, G = gridDim.x, b = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int nlive = 0;
  for (int j = 0; j < k; ++j) nlive += S.live[j];
  if (nlive == k) return true;
  long long nd = 0;
  __shared__ double s_tgt[kMaxTrials], s_excl[kMaxTrials], s_total;
  __shared__ int s_bstar[kMaxTrials], s_best;
  double* DSUM = a.part_f + (size_t)kMaxTrials * G;   // D^2 block sums region
  if (nlive > 0) {
    assign_own_rows<NP, GENERIC>(a, S, r0, nrows);
    nd += (long long)a.s * nlive;
  } else {
    const double uf = unit_double(philox_word(a.seed, (uint64_t)a.t, 1, 0, 0));
    const int i0 = (int)floor(uf * (double)a.s);
    load_cand_row(a, S, 0, i0);
    __syncthreads();
    set_centroid_row<GENERIC>(S, S.cand, 0, a.npad, a.kpad);
    if (threadIdx.x == 0) S.live[0] = 1;
    if (b == 0) {
      for (int f = threadIdx.x; f < a.npad; f += kThreads) a.C[f] = S.cand[f];
      if (threadIdx.x == 0) a.mask[0] = 1;
    }
    own_rows_to_cands(a, S, r0, nrows, 1);
    for (int i = threadIdx.x; i < nrows; i += kThreads) S.dmin[i] = S.dc[i];
    __syncthreads();
    nd += a.s;
  }
  const int R = a.rows_per_cta;
  for (int j = 0; j < k; ++j) {
    if (S.live[j]) continue;
    // (A) block sums of D^2
    const double mine = own_dmin_sum(S, nrows);
    if (threadIdx.x == 0) DSUM[b] = mine;
    if (!gb.sync()) return false;
    // (B) total, target blocks (every CTA, identical arithmetic)
    if (w == 0) {
      double carry = 0.0;
      for (int base = 0; base < G; base += 32) {
        const double v = (base + l < G) ? __ldcg(DSUM + base + l) : 0.0;
        carry += warp_sum_f64(v);
      }
      const double total = carry;
      double tgt[kMaxTrials];
      int found[kMaxTrials];
      double excl[kMaxTrials];
#pragma unroll
      for (int t = 0; t < kMaxTrials; ++t) {
        tgt[t] = t < a.trials
            ? unit_double(philox_word(a.seed, (uint64_t)a.t, 2, 0,
                                      (uint64_t)(j * a.trials + t))) * total
            : 0.0;
        found[t] = -1;
        excl[t] = 0.0;
      }
      if (total > 0.0) {
        double run = 0.0;
        int last_pos = -1;
        double last_excl = 0.0;
        for (int base = 0; base < G; base += 32) {
          const double v = (base + l < G) ? __ldcg(DSUM + base + l) : 0.0;
          double x = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += y;
          }
          const double incl = run + x;
#pragma unroll
          for (int t = 0; t < kMaxTrials; ++t) {
            if (t < a.trials && found[t] < 0) {
              const unsigned hit = __ballot_sync(0xffffffffu, base + l < G && incl > tgt[t]);
              if (hit) {
                const int ll = __ffs(hit) - 1;
                found[t] = base + ll;
                excl[t] = __shfl_sync(0xffffffffu, incl - v, ll);
              }
            }
          }
          const unsigned pos = __ballot_sync(0xffffffffu, base + l < G && v > 0.0);
          if (pos) {
            const int ll = 31 - __clz(pos);
            last_pos = base + ll;
            last_excl = __shfl_sync(0xffffffffu, incl - v, ll);
          }
          run = __shfl_sync(0xffffffffu, incl, 31);
        }
#pragma unroll
        for (int t = 0; t < kMaxTrials; ++t)
          if (t < a.trials && found[t] < 0) { found[t] = last_pos; excl[t] = last_excl; }
      }
      if (l == 0) {
        s_total = total;
#pragma unroll
        for (int t = 0; t < kMaxTrials; ++t) {
          s_tgt[t] = tgt[t];
          s_bstar[t] = found[t];
          s_excl[t] = excl[t];
        }
      }
    }
    __syncthreads();
    // the CTA that owns a target finds the row inside its block
    for (int t = 0; t < a.trials; ++t) {
      if (s_total == 0.0) {
        if (b == 0 && threadIdx.x == 0) {
          const double u = unit_double(philox_word(a.seed, (uint64_t)a.t, 2, 0,
                                                   (uint64_t)(j * a.trials + t)));
          a.ctl->cand[t] = (int)floor(u * (double)a.s);
        }
      } else if (s_bstar[t] == b && w == 0) {
        double run = s_excl[t];
        int cand = -1, lastp = -1;
        for (int base = 0; base < nrows && cand < 0; base += 32) {
          const double v = base + l < nrows ? (double)S.dmin[base + l] : 0.0;
          double x = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += y;
          }
          const double incl = run + x;
          const unsigned hit = __ballot_sync(0xffffffffu, base + l < nrows && incl > s_tgt[t]);
          if (hit) cand = base + __ffs(hit) - 1;
          const unsigned pos = __ballot_sync(0xffffffffu, base + l < nrows && v > 0.0);
          if (pos) lastp = base + 31 - __clz(pos);
          run = __shfl_sync(0xffffffffu, incl, 31);
        }
        if (cand < 0) cand = lastp;
        if (l == 0) a.ctl->cand[t] = r0 + cand;
      }
    }
    if (!gb.sync()) return false;
    // (C) potentials of the candidates
    for (int t = 0; t < a.trials; ++t) load_cand_row(a, S, t, __ldcg(a.ctl->cand + t));
    __syncthreads();
    own_rows_to_cands(a, S, r0, nrows, a.trials);
    for (int t = 0; t < a.trials; ++t) {
      double v = 0.0;
      for (int i = threadIdx.x; i < nrows; i += kThreads)
        v += (double)fminf(S.dmin[i], S.dc[t * R + i]);
      v = block_sum_f64(v, S.red);
      if (threadIdx.x == 0) a.part_f[(size_t)t * G + b] = v;
    }
    nd += (long long)a.s * a.trials;
    if (!gb.sync()) return false;
    // (D) choose the candidate with the lowest potential
    if (w == 0) {
      int best = 0;
      double bestv = 0.0;
      for (int t = 0; t < a.trials; ++t) {
        const double phi = warp_sum_array_f64(a.part_f + (size_t)t * G, G);
        if (t == 0 || phi < bestv) { bestv = phi; best = t; }
      }
      if (l == 0) s_best = best;
    }
    __syncthreads();
    const int bt = s_best;
    set_centroid_row<GENERIC>(S, S.cand + bt * a.npad, j, a.npad, a.kpad);
    if (threadIdx.x == 0) S.live[j] = 1;
    if (b == 0) {
      for (int f = threadIdx.x; f < a.npad; f += kThreads)
        a.C[(size_t)j * a.npad + f] = S.cand[bt * a.npad + f];
      if (threadIdx.x == 0) a.mask[j] = 1;
    }
    for (int i = threadIdx.x; i < nrows; i += kThreads)
      S.dmin[i] = fminf(S.dmin[i], S.dc[bt * R + i]);
    __syncthreads();
  }
  // make the reseeded rows of the global working C visible before Lloyd
  if (!gb.sync()) return false;
  *nd_out += nd;
  return true;
}

// Lloyd iterations on P (Sec. 2) with the stop rule of Sec. 5.
template <int NP, bool GENERIC>
__device__ bool phase_lloyd(const ChunkArgs& a, const Smem& S,
                            const ChunkSmem& L, GridBarrier& gb, int r0,
                            int nrows, long long* nd_out, double* f_out,
                            int* it_out) {
  const int k = a.k, n = a.n, npad = a.npad, G = gridDim.x, b = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  double* FPART = a.part_f + (size_t)(kMaxTrials + 1) * G;
  __shared__ double s_f;
  double f_prev = 0.0, f = 0.0;
  int it = 0;
  long long nd = 0;
  while (true) {
    int nlive = 0;
    for (int j = 0; j < k; ++j) nlive += S.live[j];
    assign_own_rows<NP, GENERIC>(a, S, r0, nrows);
    const double fp = own_dmin_sum(S, nrows);
    update_partials<GENERIC>(a, S, L, r0, nrows, G);
    if (threadIdx.x == 0) FPART[b] = fp;
    nd += (long long)a.s * nlive;
    if (!gb.sync()) return false;
    if (w == 0) {
      const double t = warp_sum_array_f64(FPART, G);
      if (l == 0) s_f = t;
    }
    __syncthreads();
    f = s_f;
    const bool stop = (f == 0.0) || (it > 0 && f_prev - f <= a.tol * f_prev) ||
                      (it == a.max_iter);
    const int gw = b * kWarps + w, nw = G * kWarps;
    for (int q = gw; q < k * n; q += nw) {
      const int j = q / n, ff = q - j * n;
      if (!S.live[j]) continue;
      int cnt = 0;
      for (int u = l; u < G; u += 32) cnt += __ldcg(a.part_cnt + (size_t)j * G + u);
      cnt = warp_sum_i32(cnt);
      if (cnt == 0) {
        if (ff == 0 && l == 0) a.mask[j] = 0;
        continue;
      }
      if (stop) continue;
      float sum = 0.f;
      const float* ps = a.part_sum + ((size_t)j * npad + ff) * G;
      for (int u = l; u < G; u += 32) sum += __ldcg(ps + u);
      sum = warp_sum_f32(sum);
      if (l == 0) {
        const float c = GENERIC ? S.cen[ff * a.kpad + j] : S.cen[j * npad + ff];
        a.C[(size_t)j * npad + ff] = c + sum / (float)cnt;
      }
    }
    if (!gb.sync()) return false;
    for (int j = threadIdx.x; j < k; j += kThreads)
      S.live[j] = __ldcg(reinterpret_cast<const unsigned char*>(a.mask) + j) != 0;
    if (!stop) {
      for (int q = threadIdx.x; q < k * npad; q += kThreads) {
        const int j = q / npad, ff = q - j * npad;
        const float v = __ldcg(a.C + q);
        if (GENERIC) S.cen[ff * a.kpad + j] = v;
        else S.cen[q] = v;
      }
    }
    __syncthreads();
    if (stop) break;
    f_prev = f;
    ++it;
  }
  *nd_out += nd;
  *f_out = f;
  *it_out = it;
  return true;
}

// ------------------------------------------------------------ chunk kernel
template <int NP, bool GENERIC>
__global__ void __launch_bounds__(kThreads)
chunk_kernel(ChunkArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  const int G = gridDim.x;
  const ChunkSmem L = chunk_smem(a.npad, a.k, a.kpad, a.rows_per_cta, GENERIC);
  const Smem S = carve(smem_raw, L);
  GridBarrier gb{a.ctl->bar + a.bar_sel, &a.ctl->status, 0u};
  const int r0 = min(a.s, (int)blockIdx.x * a.rows_per_cta);
  const int nrows = min(a.rows_per_cta, a.s - r0);
  long long nd = 0;
  double f = 0.0;
  int it = 0;
  bool ok = true;

  const bool full = (a.phases & kPhaseKeep) != 0;
  if (a.phases & (kPhaseKpp | kPhaseLloyd)) {
    // C' <- C (Alg. 1): the working copy starts from the incumbent.
    const float* src = full ? a.Cinc : a.C;
    const uint8_t* msrc = full ? a.mask_inc : a.mask;
    load_centroids<GENERIC>(S.cen, S.live, src, a.npad, msrc, a.k, a.n, a.npad,
                            a.kpad, true);
    if (full && blockIdx.x == 0) {
      for (int q = threadIdx.x; q < a.k * a.npad; q += kThreads) a.C[q] = __ldcg(a.Cinc + q);
      for (int j = threadIdx.x; j < a.k; j += kThreads) a.mask[j] = S.live[j];
    }
  }
  if (ok && (a.phases & kPhaseDraw)) ok = phase_draw(a, S, gb);
  if (ok && (a.phases & kPhaseGather)) {
    phase_gather(a, r0, nrows);
    ok = gb.sync();
  }
  if (ok && (a.phases & kPhaseKpp)) ok = phase_kpp<NP, GENERIC>(a, S, gb, r0, nrows, &nd);
  if (ok && (a.phases & kPhaseLloyd))
    ok = phase_lloyd<NP, GENERIC>(a, S, L, gb, r0, nrows, &nd, &f, &it);
  if (!ok) return;
  if (blockIdx.x == 0) {
    __shared__ int s_acc;
    if (threadIdx.x == 0) {
      s_acc = 0;
      if (full) s_acc = f < *a.f_opt;
      a.ctl->f_out = f;
      a.ctl->iters_out = it;
      a.ctl->bar[a.bar_sel ^ 1] = 0u;   // ready for the next launch
    }
    __syncthreads();
    if (s_acc) {
      for (int q = threadIdx.x; q < a.k * a.npad; q += kThreads) a.Cinc[q] = __ldcg(a.C + q);
      for (int j = threadIdx.x; j < a.k; j += kThreads)
        a.mask_inc[j] = __ldcg(reinterpret_cast<const unsigned char*>(a.mask) + j);
    }
    if (threadIdx.x == 0) {
      if (s_acc) *a.f_opt = f;
      if (full) {
        a.stats->chunks += 1;
        a.stats->accepted += s_acc;
        a.stats->lloyd_iters += it;
      }
      a.stats->n_d += nd;
    }
  }
  (void)G;
}

// ----------------------------------------------------------- assign kernels
__device__ __forceinline__ void assign_finish(const AssignArgs& a, double acc,
                                              double* red) {
  const double blk = block_sum_f64(acc, red);
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = blk;
    __threadfence();
    const uint32_t t = atomicAdd(a.ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x < 32) {
    __threadfence();
    const double tot = warp_sum_array_f64(a.part, gridDim.x);
    if (threadIdx.x == 0) {
      *a.sse = tot;
      *a.ticket = 0u;
    }
  }
}

template <int NP>
__global__ void __launch_bounds__(kThreads)
assign_np_kernel(AssignArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  float* cen = reinterpret_cast<float*>(smem_raw);
  int* live = reinterpret_cast<int*>(smem_raw + align_up(a.k * NP * 4, 16));
  double* red = reinterpret_cast<double*>(smem_raw + align_up(a.k * NP * 4, 16) +
                                          align_up(a.k * 4, 16));
  load_centroids<false>(cen, live, a.C, a.cstride, a.mask, a.k, a.n, NP, 0, false);
  const bool vec4 = (a.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < a.m;
       i += (long long)gridDim.x * kThreads) {
    float p[NP];
    load_row_np<NP>(p, a.X + (size_t)i * a.n, a.n, vec4, false);
    int j;
    float d;
    nearest_np<NP>(p, cen, live, a.k, j, d);
    if (a.labels) a.labels[i] = j;
    if (a.dmin) a.dmin[i] = d;
    acc += (double)d;
  }
  assign_finish(a, acc, red);
}

__global__ void __launch_bounds__(kThreads)
assign_generic_kernel(AssignArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  float* cenT = reinterpret_cast<float*>(smem_raw);
  int o = align_up(a.npad * a.kpad * 4, 16);
  int* live = reinterpret_cast<int*>(smem_raw + o);
  o += align_up(a.k * 4, 16);
  float* stage = reinterpret_cast<float*>(smem_raw + o);
  o += align_up(64 * a.npad * 4, 16);
  double* red = reinterpret_cast<double*>(smem_raw + o);
  load_centroids<true>(cenT, live, a.C, a.cstride, a.mask, a.k, a.n, a.npad, a.kpad, false);
  const bool vec4 = (a.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
  double acc = 0.0;
  const long long tiles = (a.m + 63) / 64;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long r0 = tile * 64;
    const int rows = (int)min(64LL, a.m - r0);
    stage_tile(stage, a.X + (size_t)r0 * a.n, a.n, rows, a.n, a.npad, vec4, false);
    int j;
    float d;
    if (nearest_tile(stage, cenT, live, a.k, a.kpad, a.n, rows, j, d)) {
      const long long i = r0 + (threadIdx.x >> 5) * 8 + (threadIdx.x & 31);
      if (a.labels) a.labels[i] = j;
      if (a.dmin) a.dmin[i] = d;
      acc += (double)d;
    }
    __syncthreads();
  }
  assign_finish(a, acc, red);
}

// ------------------------------------------------------------ launch glue
template <int NP, bool GENERIC>
static cudaError_t launch_chunk_t(const ChunkArgs& a, int grid, size_t smem,
                                  cudaStream_t st) {
  auto fn = chunk_kernel<NP, GENERIC>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ChunkArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kThreads),
                                     args, smem, st);
}

template <int NP, bool GENERIC>
static int chunk_max_grid_t(size_t smem) {
  auto fn = chunk_kernel<NP, GENERIC>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

cudaError_t launch_chunk(const ChunkArgs& a, int grid, bool generic, int np,
                         size_t smem, cudaStream_t st) {
  if (generic) return launch_chunk_t<0, true>(a, grid, smem, st);
  switch (np) {
    case 4: return launch_chunk_t<4, false>(a, grid, smem, st);
    case 8: return launch_chunk_t<8, false>(a, grid, smem, st);
    case 16: return launch_chunk_t<16, false>(a, grid, smem, st);
    default: return launch_chunk_t<32, false>(a, grid, smem, st);
  }
}

int chunk_max_grid(bool generic, int np, size_t smem) {
  if (generic) return chunk_max_grid_t<0, true>(smem);
  switch (np) {
    case 4: return chunk_max_grid_t<4, false>(smem);
    case 8: return chunk_max_grid_t<8, false>(smem);
    case 16: return chunk_max_grid_t<16, false>(smem);
    default: return chunk_max_grid_t<32, false>(smem);
  }
}

size_t assign_smem(int npad, int k, int kpad, bool generic) {
  if (!generic) return align_up(k * npad * 4, 16) + align_up(k * 4, 16) + 64 * 8;
  return align_up(npad * kpad * 4, 16) + align_up(k * 4, 16) +
         align_up(64 * npad * 4, 16) + 64 * 8;
}

template <typename F>
static int max_grid_of(F fn, size_t smem) {
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

int assign_max_grid(bool generic, int np, size_t smem) {
  if (generic) return max_grid_of(assign_generic_kernel, smem);
  switch (np) {
    case 4: return max_grid_of(assign_np_kernel<4>, smem);
    case 8: return max_grid_of(assign_np_kernel<8>, smem);
    case 16: return max_grid_of(assign_np_kernel<16>, smem);
    default: return max_grid_of(assign_np_kernel<32>, smem);
  }
}

cudaError_t launch_assign(const AssignArgs& a, int grid, bool generic, int np,
                          size_t smem, cudaStream_t st) {
  if (generic) {
    cudaFuncSetAttribute(assign_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    assign_generic_kernel<<<grid, kThreads, smem, st>>>(a);
  } else {
    switch (np) {
      case 4:
        cudaFuncSetAttribute(assign_np_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        assign_np_kernel<4><<<grid, kThreads, smem, st>>>(a);
        break;
      case 8:
        cudaFuncSetAttribute(assign_np_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        assign_np_kernel<8><<<grid, kThreads, smem, st>>>(a);
        break;
      case 16:
        cudaFuncSetAttribute(assign_np_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        assign_np_kernel<16><<<grid, kThreads, smem, st>>>(a);
        break;
      default:
        cudaFuncSetAttribute(assign_np_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        assign_np_kernel<32><<<grid, kThreads, smem, st>>>(a);
        break;
    }
  }
  return cudaGetLastError();
}

}  // namespace bm
