// Big-means hot path on sm_103a.
//
// chunk_kernel: one cooperative launch per chunk runs Alg. 1's loop body on
// the whole GPU -- gather P = X[idx] of the pre-drawn sample, K-means++ reseed
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
#include "bm_chunk_common.cuh"
#include "bm_kpp.cuh"
#include "bm_tile.cuh"

namespace bm {

// ---------------------------------------------------------------- smem view
struct Smem {
  float* cen;   // np: [k][npad]   generic: [npad][kpad] (transposed)
  float* crow;  // generic: [k][npad] row-major copy of the centroids
  int* live;    // [k]
  int* lidx;    // [k + 1]: live centroid indices ascending, count at [k]
  float* sw;    // generic: update accumulators [wu][k][npad]; np: label sort (ints)
  int* cw;      // generic: [wu][k] member counts; np: per-warp label counts [warps][k]
  int* lab;     // [R] labels of own rows
  float* dmin;  // [R] nearest squared distance / K-means++ D^2 of own rows
  float* dc;    // [kMaxTrials][R] candidate distances of own rows
  float* cand;  // [kMaxTrials][npad] candidate rows
  float* stage; // generic: swizzled transposed 64-row tile
  float* prow;  // np: [R][npad] own sample rows, resident for the chunk
  double* red;  // scratch for block reductions (64 doubles)
};

__device__ __forceinline__ Smem carve(char* base, const ChunkSmem& L) {
  Smem S;
  S.cen = reinterpret_cast<float*>(base + L.cen);
  S.crow = reinterpret_cast<float*>(base + L.crow);
  S.live = reinterpret_cast<int*>(base + L.live);
  S.lidx = reinterpret_cast<int*>(base + L.lidx);
  S.sw = reinterpret_cast<float*>(base + L.sw);
  S.cw = reinterpret_cast<int*>(base + L.cw);
  S.lab = reinterpret_cast<int*>(base + L.lab);
  S.dmin = reinterpret_cast<float*>(base + L.dmin);
  S.dc = reinterpret_cast<float*>(base + L.dc);
  S.cand = reinterpret_cast<float*>(base + L.cand);
  S.stage = reinterpret_cast<float*>(base + L.stage);
  S.prow = reinterpret_cast<float*>(base + L.prow);
  S.red = reinterpret_cast<double*>(base + L.red);
  return S;
}


// Centroid (j, f) into the shared tables of either layout (the tiled layout
// keeps a row-major copy too unless WITH_ROW is false).
template <bool GENERIC, bool WITH_ROW = true>
__device__ __forceinline__ void put_centroid(float* cen, float* crow, int j, int f,
                                             float v, int npad, int kpad) {
  if (GENERIC) {
    cen[f * kpad + j] = v;
    if (WITH_ROW) crow[j * npad + f] = v;
  } else {
    cen[j * npad + f] = v;
  }
}

// Centroid rows (global, k x cstride) -> shared tables; mask -> live.
template <bool GENERIC, bool WITH_ROW = true>
__device__ void load_centroids(float* cen, float* crow, int* live, const float* C,
                               int cstride, const uint8_t* mask, int k, int n,
                               int npad, int kpad, bool coherent) {
  for (int q = threadIdx.x; q < k * npad; q += blockDim.x) {
    const int j = q / npad, f = q - j * npad;
    float v = 0.f;
    if (f < n) v = coherent ? __ldcg(C + (size_t)j * cstride + f)
                            : __ldg(C + (size_t)j * cstride + f);
    put_centroid<GENERIC, WITH_ROW>(cen, crow, j, f, v, npad, kpad);
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const unsigned char mv = coherent
        ? __ldcg(reinterpret_cast<const unsigned char*>(mask) + j)
        : __ldg(reinterpret_cast<const unsigned char*>(mask) + j);
    live[j] = mv != 0;
  }
  __syncthreads();
}

// ------------------------------------------------------------ np path rows
// Row of n floats (zero padded to NP) from global memory into registers.
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

// Row of NP floats from shared memory (16-byte aligned) into registers.
template <int NP>
__device__ __forceinline__ void load_row_smem(float (&p)[NP], const float* row) {
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const float4 v = reinterpret_cast<const float4*>(row)[q];
    p[4 * q] = v.x; p[4 * q + 1] = v.y; p[4 * q + 2] = v.z; p[4 * q + 3] = v.w;
  }
}

// Squared distances of two register-held rows to a register-held centroid
// row c.  Each row keeps four independent partial sums (features f mod 4),
// combined as (s0 + s1) + (s2 + s3).
template <int NP>
__device__ __forceinline__ void dist2_np(const float (&pa)[NP], const float (&pb)[NP],
                                         const float4 (&c)[NP / 4], float& da, float& db) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  float b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
#pragma unroll
  for (int u = 0; u < NP / 4; ++u) {
    const float4 v = c[u];
    a0 = sq(pa[4 * u] - v.x, a0);
    a1 = sq(pa[4 * u + 1] - v.y, a1);
    a2 = sq(pa[4 * u + 2] - v.z, a2);
    a3 = sq(pa[4 * u + 3] - v.w, a3);
    b0 = sq(pb[4 * u] - v.x, b0);
    b1 = sq(pb[4 * u + 1] - v.y, b1);
    b2 = sq(pb[4 * u + 2] - v.z, b2);
    b3 = sq(pb[4 * u + 3] - v.w, b3);
  }
  da = (a0 + a1) + (a2 + a3);
  db = (b0 + b1) + (b2 + b3);
}

// Nearest centroid among live-list positions [q0, q1) for two rows, in
// ascending index order with strict <; a label stays out of range when the
// range holds no centroid.  The next centroid's row is loaded from shared
// memory while the current one is scored, so the loads' latency overlaps
// the arithmetic.
template <int NP>
__device__ __forceinline__ void nearest2_np(const float (&pa)[NP], const float (&pb)[NP],
                                            const float* cen, const int* lidx, int q0,
                                            int q1, int& ja, float& da, int& jb,
                                            float& db) {
  da = db = INFINITY;
  ja = jb = INT_MAX;
  if (q0 >= q1) return;
  float4 cv[NP / 4];
  int j = lidx[q0];
#pragma unroll
  for (int u = 0; u < NP / 4; ++u) cv[u] = reinterpret_cast<const float4*>(cen + j * NP)[u];
#pragma unroll 1
  for (int q = q0; q < q1; ++q) {
    const int jn = lidx[min(q + 1, q1 - 1)];   // the last step reloads its own row
    float4 nv[NP / 4];
#pragma unroll
    for (int u = 0; u < NP / 4; ++u) nv[u] = reinterpret_cast<const float4*>(cen + jn * NP)[u];
    float d0, d1;
    dist2_np<NP>(pa, pb, cv, d0, d1);
    if (ja == INT_MAX || d0 < da) { da = d0; ja = j; }
    if (jb == INT_MAX || d1 < db) { db = d1; jb = j; }
#pragma unroll
    for (int u = 0; u < NP / 4; ++u) cv[u] = nv[u];
    j = jn;
  }
}

// Nearest live centroid of every own row (resident in S.prow) -> S.lab /
// S.dmin.  The shared-memory reads of the
// centroid table, not the arithmetic, limit a one-row-per-thread scan, so
// each thread takes two rows and each half of the CTA scans one half of the
// live list: the lower half writes its winners to S.lab / S.dmin, the upper
// half to `spare` ([R] distances, then [R] labels), and the halves merge in
// index order -- the upper half's winner replaces the lower's only when
// strictly nearer (or when the lower half found none), so the lowest index
// still wins ties.  With SUM, the merge also starts the fixed-order sum of
// the rows' distances (dmin_sum's arithmetic): each warp's exact FP32 pair
// goes to S.red[warp] as a double, for lloyd_own_rows to add up.
static_assert(kMaxTrials >= 2, "nearest_own_rows keeps 2 x R words in S.dc");

template <int NP, bool SUM>
__device__ void nearest_own_rows(const Smem& S, float* spare, int R, int k, int nrows) {
  const int H = blockDim.x >> 1;
  const bool upper = threadIdx.x >= H;
  const int u = threadIdx.x - (upper ? H : 0);
  const int nl = S.lidx[k], h = (nl + 1) >> 1;
  const int q0 = upper ? h : 0, q1 = upper ? nl : h;
  int* spare_lab = reinterpret_cast<int*>(spare + R);
  for (int base = 0; base < nrows; base += 2 * H) {
    const int ia = base + u, ib = base + H + u;
    if (ia >= nrows) break;
    float pa[NP], pb[NP];
    load_row_smem<NP>(pa, S.prow + ia * NP);
    load_row_smem<NP>(pb, S.prow + (ib < nrows ? ib : ia) * NP);
    int ja, jb;
    float da, db;
    nearest2_np<NP>(pa, pb, S.cen, S.lidx, q0, q1, ja, da, jb, db);
    if (upper) {
      spare[ia] = da;
      spare_lab[ia] = ja;
      if (ib < nrows) { spare[ib] = db; spare_lab[ib] = jb; }
    } else {
      S.dmin[ia] = da;
      S.lab[ia] = ja;
      if (ib < nrows) { S.dmin[ib] = db; S.lab[ib] = jb; }
    }
  }
  __syncthreads();
  float hi = 0.f, lo = 0.f;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    const float dh = spare[i];
    float d = S.dmin[i];
    if (S.lab[i] == INT_MAX || dh < d) {
      d = dh;
      S.dmin[i] = dh;
      S.lab[i] = spare_lab[i];
    }
    if (SUM) two_sum_acc(hi, lo, d);
  }
  if (SUM) {
    warp_two_sum(hi, lo);
    if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = (double)hi + (double)lo;
  }
  __syncthreads();
}

// -------------------------------------------------------- generic path rows
// ------------------------------------------------------ own-row helpers
// Own sample rows -> the resident shared copy (row-in-register path), when
// P was written by the host rather than by this launch's gather.
template <int NP>
__device__ void stage_own_rows(const ChunkArgs& a, const Smem& S, int r0, int nrows) {
  const int nq = NP / 4;
  for (int e = threadIdx.x; e < nrows * nq; e += blockDim.x) {
    const int i = e / nq, q = e - i * nq;
    reinterpret_cast<float4*>(S.prow + i * NP)[q] =
        __ldcg(reinterpret_cast<const float4*>(a.P + (size_t)(r0 + i) * NP) + q);
  }
  __syncthreads();
}

// Nearest live centroid of every own row -> S.lab / S.dmin.
template <int NP, bool GENERIC>
__device__ void assign_own_rows(const ChunkArgs& a, const Smem& S, int r0,
                                int nrows) {
  if constexpr (!GENERIC) {
    nearest_own_rows<NP, false>(S, S.dc, a.rows_per_cta, a.k, nrows);
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

// Fixed-order sum of S.dmin over own rows (see dmin_sum); every thread gets it.
__device__ __forceinline__ double own_dmin_sum(const Smem& S, int nrows) {
  return dmin_sum(S.dmin, nrows, S.red);
}

// Squared distances of own rows to the nc candidate rows in S.cand
// -> S.dc[c][i].
template <int NP, bool GENERIC>
__device__ void own_rows_to_cands(const ChunkArgs& a, const Smem& S, int r0,
                                  int nrows, int nc) {
  const int R = a.rows_per_cta, npad = a.npad;
  if constexpr (!GENERIC) {
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      float p[NP];
      load_row_smem<NP>(p, S.prow + i * NP);
      for (int c = 0; c < nc; ++c) {
        const float4* c4 = reinterpret_cast<const float4*>(S.cand + c * npad);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int u = 0; u < NP / 4; ++u) {
          const float4 v = c4[u];
          s0 = sq(p[4 * u] - v.x, s0);
          s1 = sq(p[4 * u + 1] - v.y, s1);
          s2 = sq(p[4 * u + 2] - v.z, s2);
          s3 = sq(p[4 * u + 3] - v.w, s3);
        }
        S.dc[c * R + i] = (s0 + s1) + (s2 + s3);
      }
    }
    __syncthreads();
  } else {
    for (int t0 = 0; t0 < nrows; t0 += 64) {
      const int rows = min(64, nrows - t0);
      stage_tile(S.stage, a.P + (size_t)(r0 + t0) * npad, npad, rows, a.n, npad,
                 true, true);
      for (int e = threadIdx.x; e < 64 * nc; e += blockDim.x) {
        const int r = e & 63, c = e >> 6;
        const float* cr = S.cand + c * npad;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int f = 0;
        for (; f + 4 <= a.n; f += 4) {
          s0 = sq(S.stage[f * 64 + (r ^ swz(f))] - cr[f], s0);
          s1 = sq(S.stage[(f + 1) * 64 + (r ^ swz(f + 1))] - cr[f + 1], s1);
          s2 = sq(S.stage[(f + 2) * 64 + (r ^ swz(f + 2))] - cr[f + 2], s2);
          s3 = sq(S.stage[(f + 3) * 64 + (r ^ swz(f + 3))] - cr[f + 3], s3);
        }
        for (; f < a.n; ++f) s0 = sq(S.stage[f * 64 + (r ^ swz(f))] - cr[f], s0);
        if (r < rows) S.dc[c * R + t0 + r] = (s0 + s1) + (s2 + s3);
      }
      __syncthreads();
    }
  }
}

// One Lloyd assignment over own rows plus the partial sums of the update:
// S.lab / S.dmin, part_sum[j][f][b] = sum over own rows labelled j of
// (p_f - c_jf) and part_cnt[j][b], and (thread 0's *fp) the fixed-order sum
// of the rows' distances, dmin_sum's value.  Every sum has a fixed order.
//   np path: a stable counting sort of the rows by label, then thread
//            (j, f) adds centroid j's rows in row order;
//   generic: per row-group accumulators [k][npad], thread = (group, feature),
//            rows of each staged tile split among the groups.
template <int NP, bool GENERIC>
__device__ void lloyd_own_rows(const ChunkArgs& a, const Smem& S,
                               const ChunkSmem& L, int r0, int nrows, int G, double* fp) {
  const int k = a.k, n = a.n, npad = a.npad, b = blockIdx.x;
  if constexpr (!GENERIC) {
    uint64_t tsub = trace_now(a);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    (void)L;
    // assignment (S.dc, the K-means++ candidate distances, is free here)
    nearest_own_rows<NP, true>(S, S.dc, a.rows_per_cta, k, nrows);
    phase_tick(a, 8, &tsub);
    // stable counting sort of own rows by label: order[start[j] ..) lists
    // centroid j's rows in ascending row order
    int* order = reinterpret_cast<int*>(S.sw);
    int* start = order + a.rows_per_cta;   // [k + 1]
    int* cur = start + k + 1;              // [k]
    int* wc = S.cw;                        // [warps][k]
    for (int j = threadIdx.x; j < k; j += blockDim.x) cur[j] = 0;
    for (int q = threadIdx.x; q < nw * k; q += blockDim.x) wc[q] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      const int j = S.lab[i];
      if (j < k) atomicAdd(cur + j, 1);
    }
    __syncthreads();
    if (w == 0) {
      int run = 0;
      for (int base = 0; base < k; base += 32) {
        const int j = base + l;
        const int c = j < k ? cur[j] : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (l >= o) x += y;
        }
        if (j < k) start[j] = run + x - c;
        run += __shfl_sync(0xffffffffu, x, 31);
      }
      if (l == 0) start[k] = run;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) cur[j] = start[j];
    __syncthreads();
    for (int i0 = 0; i0 < nrows; i0 += blockDim.x) {
      const int i = i0 + threadIdx.x;
      int j = i < nrows ? S.lab[i] : k;
      if (j > k) j = k;
      const unsigned peers = __match_any_sync(0xffffffffu, j);
      const int rank = __popc(peers & ((1u << l) - 1u));
      if (j < k && rank == 0) wc[w * k + j] = __popc(peers);
      __syncthreads();
      if (j < k) {
        int pos = cur[j] + rank;
        for (int u = 0; u < w; ++u) pos += wc[u * k + j];
        order[pos] = i;
      }
      __syncthreads();
      for (int jj = threadIdx.x; jj < k; jj += blockDim.x) {
        int add = 0;
        for (int u = 0; u < nw; ++u) {
          add += wc[u * k + jj];
          wc[u * k + jj] = 0;
        }
        cur[jj] += add;
      }
      __syncthreads();
    }
    phase_tick(a, 9, &tsub);
    // partial sums of (p - c_j) over each centroid's rows, in row order;
    // thread (j, q) keeps the four chains of features 4q .. 4q + 3 (one
    // float4 load per row), so k * NP / 4 threads cover the table in one
    // round.  Padding features sum exact zeros.
    constexpr int NQ = NP / 4;
    for (int t = threadIdx.x; t < k * NQ; t += blockDim.x) {
      const int j = t / NQ, qd = t - j * NQ;
      if (4 * qd >= n) continue;
      const float4 c = reinterpret_cast<const float4*>(S.cen + j * NP)[qd];
      const int e0 = start[j], e1 = start[j + 1];
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
      for (int e = e0; e < e1; ++e) {
        const float4 v = reinterpret_cast<const float4*>(S.prow + order[e] * NP)[qd];
        s0 += v.x - c.x;
        s1 += v.y - c.y;
        s2 += v.z - c.z;
        s3 += v.w - c.w;
      }
      float* ps = a.part_sum + ((size_t)j * npad + 4 * qd) * G + b;
      ps[0] = s0;
      ps[(size_t)G] = s1;
      ps[2 * (size_t)G] = s2;
      ps[3 * (size_t)G] = s3;
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      if (BM_GUARD(j < a.k, &a.ctl->status)) a.part_cnt[(size_t)j * G + b] = start[j + 1] - start[j];
    __syncthreads();
    if (threadIdx.x == 0) {   // the merge left one exact pair per warp in S.red
      double t = 0.0;
      for (int i = 0; i < nw; ++i) t += S.red[i];
      *fp = t;
    }
    phase_tick(a, 10, &tsub);
  } else {
    const int ng = L.wu;
    for (int q = threadIdx.x; q < ng * k * npad; q += blockDim.x) S.sw[q] = 0.f;
    for (int q = threadIdx.x; q < ng * k; q += blockDim.x) S.cw[q] = 0;
    for (int t0 = 0; t0 < nrows; t0 += 64) {
      const int rows = min(64, nrows - t0);
      stage_tile(S.stage, a.P + (size_t)(r0 + t0) * npad, npad, rows, n, npad, true, true);
      int j;
      float d;
      if (nearest_tile(S.stage, S.cen, S.live, k, a.kpad, n, rows, j, d)) {
        const int i = t0 + (threadIdx.x >> 5) * 8 + (threadIdx.x & 31);
        S.lab[i] = j;
        S.dmin[i] = d;
      }
      __syncthreads();
      for (int slot = threadIdx.x; slot < ng * npad; slot += blockDim.x) {
        const int g = slot / npad, f = slot - g * npad;
        if (f >= n) continue;
        float* acc = S.sw + g * k * npad;
        const int sz = swz(f);
        for (int r = g; r < rows; r += ng) {
          const int jr = S.lab[t0 + r];
          if (jr >= k) continue;
          acc[jr * npad + f] += S.stage[f * 64 + (r ^ sz)] - S.crow[jr * npad + f];
          if (f == 0) S.cw[g * k + jr] += 1;
        }
      }
      __syncthreads();
    }
    for (int q = threadIdx.x; q < k * npad; q += blockDim.x) {
      const int jj = q / npad, f = q - jj * npad;
      if (f < n) {
        float sum = 0.f;
        for (int g = 0; g < ng; ++g) sum += S.sw[g * k * npad + q];
        if (BM_GUARD(jj < a.k && f < npad, &a.ctl->status))
          a.part_sum[((size_t)jj * npad + f) * G + b] = sum;
      }
    }
    for (int jj = threadIdx.x; jj < k; jj += blockDim.x) {
      int c = 0;
      for (int g = 0; g < ng; ++g) c += S.cw[g * k + jj];
      if (BM_GUARD(jj < a.k, &a.ctl->status)) a.part_cnt[(size_t)jj * G + b] = c;
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
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) {
    if (i < w) before += buf[i];
    all += buf[i];
  }
  *total = all;
  return before + x - v;
}

// ------------------------------------------------------------------ phases
// P[i] = X[idx[i]] for own rows (zero padding to npad).  The row-in-register
// path gathers one row per thread with independent vector loads and also
// keeps the row in the CTA's resident copy; the tiled path copies elements,
// eight independent loads in flight per thread.
template <int NP, bool GENERIC>
__device__ void phase_gather(const ChunkArgs& a, const Smem& S, int r0, int nrows) {
  const int npad = a.npad, n = a.n;
  const long long ready = gather_rows_ready(a, r0, nrows);
  if constexpr (!GENERIC) {
    const bool vec4 = (n % 4 == 0) && gather_sources_aligned16(a);
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      long long row = __ldcg(a.idx + r0 + i);
      if (!BM_GUARD(row >= 0 && row < a.m, &a.ctl->status)) row = 0;
      float p[NP];
      load_row_np<NP>(p, gather_row_source(a, row, ready) + (size_t)row * n, n, vec4, false);
      float4* dst = reinterpret_cast<float4*>(a.P + (size_t)(r0 + i) * NP);
      float4* res = reinterpret_cast<float4*>(S.prow + i * NP);
#pragma unroll
      for (int q = 0; q < NP / 4; ++q) {
        const float4 v = make_float4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
        dst[q] = v;
        res[q] = v;
      }
    }
  } else {
    const int total = nrows * npad;
    for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = 0.f;
        if (e < total) {
          const int i = e / npad, f = e - i * npad;
          const long long row = __ldcg(a.idx + r0 + i);
          if (f < n && BM_GUARD(row >= 0 && row < a.m, &a.ctl->status))
            v[u] = __ldg(gather_row_source(a, row, ready) + (size_t)row * n + f);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total) a.P[(size_t)r0 * npad + e] = v[u];
      }
    }
  }
  __syncthreads();
}

template <bool GENERIC>
__device__ __forceinline__ void set_centroid_row(const Smem& S, const float* src,
                                                 int j, int npad, int kpad) {
  for (int f = threadIdx.x; f < npad; f += blockDim.x)
    put_centroid<GENERIC>(S.cen, S.crow, j, f, src[f], npad, kpad);
}

__device__ __forceinline__ void load_cand_row(const ChunkArgs& a, const Smem& S,
                                              int c, int row) {
  if (!BM_GUARD(row >= 0 && row < a.s, &a.ctl->status)) row = 0;
  for (int f = threadIdx.x; f < a.npad; f += blockDim.x)
    S.cand[c * a.npad + f] = __ldcg(a.P + (size_t)row * a.npad + f);
}

// Forgy's row for slot j: floor(u_j * s), u_j the slot's first K-means++
// uniform.
__device__ __forceinline__ int forgy_row(const ChunkArgs& a, int j) {
  const double u = unit_double(philox_word(a.seed, (uint64_t)a.t, 2, 0,
                                           (uint64_t)(j * a.trials)));
  return min(a.s - 1, (int)floor(u * (double)a.s));
}

// CTA 0: sample row `row` -> slot j of the global working C (the same
// L2-coherent loads that fill the candidate table, so the same bits).
__device__ __forceinline__ void put_global_row(const ChunkArgs& a, int j, int row) {
  for (int f = threadIdx.x; f < a.npad; f += blockDim.x)
    a.C[(size_t)j * a.npad + f] = __ldcg(a.P + (size_t)row * a.npad + f);
}

// K-means++ reseed of every degenerate slot, ascending (Sec. 3.3, Sec. 5).
//
// Without the incumbent copy (step-level calls) every CTA reads the starting
// centroids and mask from the global working C at its start.  Slots filled
// before the launch's first grid barrier -- the uniform first pick, Forgy's
// picks -- therefore reach the global C and mask only after that barrier:
// a CTA that started late would otherwise find a slot live in the mask while
// its row is still (partly) unwritten, and compute its D^2 against the wrong
// point.
template <int NP, bool GENERIC>
__device__ bool phase_kpp(const ChunkArgs& a, const Smem& S, GridBarrier& gb,
                          int r0, int nrows, long long* nd_out, unsigned long long gen) {
  const int k = a.k, G = gridDim.x, b = blockIdx.x;
  const int nlive = S.lidx[k];
  if (nlive == k) return true;
  if (a.init == kInitForgy) {
    // Forgy: slot j <- sample row floor(u_j * s); no distances, every CTA
    // applies the same picks
    for (int j = 0; j < k; ++j) {
      if (S.live[j]) continue;
      load_cand_row(a, S, 0, forgy_row(a, j));
      __syncthreads();
      set_centroid_row<GENERIC>(S, S.cand, j, a.npad, a.kpad);
      if (threadIdx.x == 0) S.live[j] = 1;
      __syncthreads();
    }
    build_live_list(S.live, S.lidx, k);
    if (!gb.sync()) return false;
    if (b == 0) {
      // the global mask still holds the starting live set: only CTA 0
      // writes it, and only below, after every row is in place
      for (int j = 0; j < k; ++j)
        if (__ldcg(reinterpret_cast<const unsigned char*>(a.mask) + j) == 0)
          put_global_row(a, j, forgy_row(a, j));
      __syncthreads();
      for (int j = threadIdx.x; j < k; j += blockDim.x) a.mask[j] = 1;
    }
    return true;
  }
  long long nd = 0;
  double* DSUM = a.part_f + (size_t)kMaxTrials * G;   // D^2 block sums region
  int first_row = -1;   // the uniform first pick, until CTA 0 has published it
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
    first_row = i0;
    own_rows_to_cands<NP, GENERIC>(a, S, r0, nrows, 1);
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) S.dmin[i] = S.dc[i];
    __syncthreads();
    nd += a.s;
  }
  // after a grid barrier: slot 0 <- the first pick in the global C and mask
  auto publish_first = [&]() {
    if (first_row < 0) return;
    if (b == 0) {
      put_global_row(a, 0, first_row);
      if (threadIdx.x == 0) a.mask[0] = 1;
    }
    first_row = -1;
  };
  const int R = a.rows_per_cta;
  __shared__ int s_rows[kMaxTrials];
  for (int j = 0; j < k; ++j) {
    if (S.live[j]) continue;
    const unsigned long long tag = kx_tag(gen, j);
    // (A) block sums of D^2
    const double mine = own_dmin_sum(S, nrows);
    kpp_put_dsum(a, DSUM, mine, tag);
    if (!gb.sync()) return false;
    publish_first();
    // (B) targets, the blocks that hold them and the rows inside those blocks
    if (!kpp_locate(a, S.dmin, r0, nrows, DSUM, j, tag)) return false;
    if (!gb.sync()) return false;
    // (C) potentials of the candidates
    if (!kpp_get_cands(a, s_rows, tag)) return false;
    for (int t = 0; t < a.trials; ++t) load_cand_row(a, S, t, s_rows[t]);
    __syncthreads();
    own_rows_to_cands<NP, GENERIC>(a, S, r0, nrows, a.trials);
    double pot[kMaxTrials];
    for (int t = 0; t < a.trials; ++t) {
      double v = 0.0;
      for (int i = threadIdx.x; i < nrows; i += blockDim.x)
        v += (double)fminf(S.dmin[i], S.dc[t * R + i]);
      pot[t] = block_sum_f64(v, S.red);
    }
    kpp_put_potentials(a, pot, tag);
    nd += (long long)a.s * a.trials;
    if (!gb.sync()) return false;
    // (D) choose the candidate with the lowest potential
    const int bt = kpp_best(a, tag);
    if (bt < 0) return false;
    set_centroid_row<GENERIC>(S, S.cand + bt * a.npad, j, a.npad, a.kpad);
    if (threadIdx.x == 0) S.live[j] = 1;
    if (b == 0) {
      for (int f = threadIdx.x; f < a.npad; f += blockDim.x)
        a.C[(size_t)j * a.npad + f] = S.cand[bt * a.npad + f];
      if (threadIdx.x == 0) a.mask[j] = 1;
    }
    for (int i = threadIdx.x; i < nrows; i += blockDim.x)
      S.dmin[i] = fminf(S.dmin[i], S.dc[bt * R + i]);
    __syncthreads();
  }
  build_live_list(S.live, S.lidx, k);
  // make the reseeded rows of the global working C visible before Lloyd
  // (Lloyd reads it back only after its own barriers, so the first pick of a
  // launch that reseeded no other slot may follow this one)
  if (!gb.sync()) return false;
  publish_first();
  *nd_out += nd;
  return true;
}

// Lloyd iterations on P (Sec. 2) with the stop rule of Sec. 5.
template <int NP, bool GENERIC>
__device__ bool phase_lloyd(const ChunkArgs& a, const Smem& S,
                            const ChunkSmem& L, GridBarrier& gb, int r0,
                            int nrows, long long* nd_out, double* f_out,
                            int* it_out, uint64_t* tclk) {
  const int k = a.k, n = a.n, npad = a.npad, G = gridDim.x, b = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  double* FPART = a.part_f + (size_t)(kMaxTrials + 1) * G;
  __shared__ double s_f;
  double f_prev = 0.0, f = 0.0;
  int it = 0;
  long long nd = 0;
  while (true) {
    const int nlive = S.lidx[k];
    double fp = 0.0;
    lloyd_own_rows<NP, GENERIC>(a, S, L, r0, nrows, G, &fp);
    if constexpr (GENERIC) fp = own_dmin_sum(S, nrows);
    if (threadIdx.x == 0) FPART[b] = fp;
    nd += (long long)a.s * nlive;
    phase_tick(a, 3, tclk);
    if (!gb.sync()) return false;
    phase_tick(a, 4, tclk);
    // Centroid (j, f) of the update belongs to warp q of the grid.  Its
    // member count and partial sums over the CTAs are fetched before the
    // stop decision (which only gates the write), and warp 0 fetches the
    // objective's partials at the same time, so the whole step costs about
    // one round trip to L2.
    const int nwb = blockDim.x >> 5;
    const int gw = b * nwb + w, nw = G * nwb;
    const int q1st = gw < k * n ? gw : -1;   // the common case: one (j, f) per warp
    int cnt1 = 0;
    float sum1 = 0.f;
    {
      const int j1 = q1st >= 0 ? q1st / n : 0, f1 = q1st >= 0 ? q1st - j1 * n : 0;
      const bool item = q1st >= 0 && S.live[j1] != 0;
      const int* pc = a.part_cnt + (size_t)j1 * G;
      const float* ps = a.part_sum + ((size_t)j1 * npad + f1) * G;
      if (G <= 256) {
        // one batch of loads: the item's counts and sums, and (warp 0) the
        // objective's partials; each lane adds its terms in CTA order
        int tc[8];
        float ts[8];
        double tf[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = 32 * u + l;
          tc[u] = item && i < G ? __ldcg(pc + i) : 0;
          ts[u] = item && i < G ? __ldcg(ps + i) : 0.f;
          tf[u] = w == 0 && i < G ? __ldcg(FPART + i) : 0.0;
        }
        double fl = 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          cnt1 += tc[u];
          sum1 += ts[u];
          fl += tf[u];
        }
        cnt1 = warp_sum_i32(cnt1);
        sum1 = warp_sum_f32(sum1);
        fl = warp_sum_f64(fl);
        if (w == 0 && l == 0) s_f = fl;
      } else {
        if (item) {
          cnt1 = warp_sum_i32(lane_sum_ldcg(pc, G));
          sum1 = warp_sum_f32(lane_sum_ldcg(ps, G));
        }
        if (w == 0) {
          const double t = warp_sum_array_f64(FPART, G);
          if (l == 0) s_f = t;
        }
      }
    }
    __syncthreads();
    f = s_f;
    const bool stop = (f == 0.0) || (it > 0 && f_prev - f <= a.tol * f_prev) ||
                      (it == a.max_iter);
    for (int q = gw; q < k * n; q += nw) {
      const int j = q / n, ff = q - j * n;
      if (!S.live[j]) continue;
      int cnt;
      float sum;
      if (q == q1st) {
        cnt = cnt1;
        sum = sum1;
      } else {
        cnt = warp_sum_i32(lane_sum_ldcg(a.part_cnt + (size_t)j * G, G));
        sum = warp_sum_f32(lane_sum_ldcg(a.part_sum + ((size_t)j * npad + ff) * G, G));
      }
      if (cnt == 0) {   // degenerate (Sec. 3.3), or kept in place and live
        if (!a.empty_keep && ff == 0 && l == 0) a.mask[j] = 0;
        continue;
      }
      if (stop) continue;
      if (l == 0) {
        const float c = GENERIC ? S.crow[j * npad + ff] : S.cen[j * npad + ff];
        a.C[(size_t)j * npad + ff] = c + sum / (float)cnt;
      }
    }
    phase_tick(a, 5, tclk);
    if (!gb.sync()) return false;
    // the new centroids and mask: four centroid values per thread and step,
    // all loads of a step in flight together
    if (!stop) {
      const int kn = k * npad, T = blockDim.x;
      for (int q0 = threadIdx.x; q0 < kn; q0 += 4 * T) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = q0 + u * T < kn ? __ldcg(a.C + q0 + u * T) : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * T;
          if (q < kn) put_centroid<GENERIC>(S.cen, S.crow, q / npad, q % npad, v[u], npad, a.kpad);
        }
      }
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      S.live[j] = __ldcg(reinterpret_cast<const unsigned char*>(a.mask) + j) != 0;
    build_live_list(S.live, S.lidx, k);
    phase_tick(a, 6, tclk);
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
__global__ void __launch_bounds__(GENERIC ? 256 : 384)
chunk_kernel(ChunkArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  BM_POISON_SMEM();
  BM_START_SKEW();
  const int G = gridDim.x;
  const ChunkSmem L = chunk_smem(a.npad, a.k, a.kpad, a.rows_per_cta, GENERIC);
  const Smem S = carve(smem_raw, L);
  GridBarrier gb{a.ctl->bar + a.bar_sel, &a.ctl->status, 0u};
  const unsigned long long gen = kx_generation(a);
  const int r0 = min(a.s, (int)blockIdx.x * a.rows_per_cta);
  const int nrows = min(a.rows_per_cta, a.s - r0);
  long long nd = 0;
  double f = 0.0;
  int it = 0;
  bool ok = true;

  if (threadIdx.x < kNumPhaseTimers) phase_slots()[threadIdx.x] = 0ull;
  uint64_t tclk = trace_now(a);
  const bool full = (a.phases & kPhaseKeep) != 0;
  if (a.phases & (kPhaseKpp | kPhaseLloyd)) {
    // C' <- C (Alg. 1): the working copy starts from the incumbent.
    const float* src = full ? a.Cinc : a.C;
    const uint8_t* msrc = full ? a.mask_inc : a.mask;
    load_centroids<GENERIC>(S.cen, S.crow, S.live, src, a.npad, msrc, a.k, a.n,
                            a.npad, a.kpad, true);
    build_live_list(S.live, S.lidx, a.k);
    if (full && blockIdx.x == 0) {
      for (int q = threadIdx.x; q < a.k * a.npad; q += blockDim.x) a.C[q] = __ldcg(a.Cinc + q);
      for (int j = threadIdx.x; j < a.k; j += blockDim.x) a.mask[j] = S.live[j];
    }
  }
  phase_tick(a, 0, &tclk);
  if (ok && (a.phases & kPhaseGather)) {
    phase_gather<NP, GENERIC>(a, S, r0, nrows);
    // Only K-means++ reads sample rows gathered by other CTAs; Lloyd reads
    // its own rows, so without a reseed no grid barrier is needed here.
    const bool reseed = (a.phases & kPhaseKpp) && S.lidx[a.k] < a.k;
    if (reseed) ok = gb.sync();
    phase_tick(a, 1, &tclk);
  } else if (a.phases & (kPhaseKpp | kPhaseLloyd)) {
    if constexpr (!GENERIC) stage_own_rows<NP>(a, S, r0, nrows);   // P written by the host
  }
  if (ok && (a.phases & kPhaseKpp)) {
    ok = phase_kpp<NP, GENERIC>(a, S, gb, r0, nrows, &nd, gen);
    phase_tick(a, 2, &tclk);
  }
  if (ok && (a.phases & kPhaseLloyd))
    ok = phase_lloyd<NP, GENERIC>(a, S, L, gb, r0, nrows, &nd, &f, &it, &tclk);
  if (!ok) return;
  if (blockIdx.x == 0) {
    __shared__ int s_acc;
    if (threadIdx.x == 0) {
      s_acc = 0;
      if (full) s_acc = f < *a.f_opt;
      a.ctl->f_out = f;
      a.ctl->iters_out = it;
      a.ctl->bar[a.bar_sel ^ 1] = 0u;   // ready for the next launch
      kx_advance(a, gen);
    }
    __syncthreads();
    if (s_acc) {
      for (int q = threadIdx.x; q < a.k * a.npad; q += blockDim.x) a.Cinc[q] = __ldcg(a.C + q);
      for (int j = threadIdx.x; j < a.k; j += blockDim.x)
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
    phase_tick(a, 7, &tclk);
    if (threadIdx.x == 0)
      for (int i = 0; i < kNumPhaseTimers; ++i) a.stats->phase_ns[i] += phase_slots()[i];
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
  BM_POISON_SMEM();
  float* cen = reinterpret_cast<float*>(smem_raw);
  int o = align_up(a.k * NP * 4, 16);
  int* live = reinterpret_cast<int*>(smem_raw + o);
  o += align_up(a.k * 4, 16);
  int* lidx = reinterpret_cast<int*>(smem_raw + o);
  o += align_up((a.k + 1) * 4, 16);
  double* red = reinterpret_cast<double*>(smem_raw + o);
  load_centroids<false>(cen, nullptr, live, a.C, a.cstride, a.mask, a.k, a.n, NP, 0, false);
  build_live_list(live, lidx, a.k);
  const bool vec4 = (a.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
  // two rows per thread, a grid stride apart: each centroid load from
  // shared memory serves both
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.m;
       i += 2 * stride) {
    const long long i2 = i + stride;
    const bool two = i2 < a.m;
    float pa[NP], pb[NP];
    load_row_np<NP>(pa, a.X + (size_t)i * a.n, a.n, vec4, false);
    load_row_np<NP>(pb, a.X + (size_t)(two ? i2 : i) * a.n, a.n, vec4, false);
    int ja, jb;
    float da, db;
    nearest2_np<NP>(pa, pb, cen, lidx, 0, lidx[a.k], ja, da, jb, db);
    if (BM_GUARD(i < a.m, a.status)) {
      if (a.labels) a.labels[i] = ja;
      if (a.dmin) a.dmin[i] = da;
    }
    acc += (double)da;
    if (two) {
      if (a.labels) a.labels[i2] = jb;
      if (a.dmin) a.dmin[i2] = db;
      acc += (double)db;
    }
  }
  assign_finish(a, acc, red);
}

__global__ void __launch_bounds__(kThreads)
assign_generic_kernel(AssignArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  BM_POISON_SMEM();
  float* cenT = reinterpret_cast<float*>(smem_raw);
  int o = align_up(a.npad * a.kpad * 4, 16);
  int* live = reinterpret_cast<int*>(smem_raw + o);
  o += align_up(a.k * 4, 16);
  float* stage = reinterpret_cast<float*>(smem_raw + o);
  o += align_up(64 * a.npad * 4, 16);
  double* red = reinterpret_cast<double*>(smem_raw + o);
  load_centroids<true, false>(cenT, nullptr, live, a.C, a.cstride, a.mask, a.k, a.n,
                              a.npad, a.kpad, false);
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
      if (BM_GUARD(i < a.m && i < r0 + rows, a.status)) {
        if (a.labels) a.labels[i] = j;
        if (a.dmin) a.dmin[i] = d;
      }
      acc += (double)d;
    }
    __syncthreads();
  }
  assign_finish(a, acc, red);
}

// Publishes that the first `count` pieces of X have landed: the
// host-to-device copies of those pieces precede it on its stream.  Chunk
// gathers read the rows of landed pieces from X, the others from the host
// copy.
__global__ void x_ready_kernel(uint32_t* landed, uint32_t count) {
  __threadfence();
  atomicMax(landed, count);
}

// ------------------------------------------------------------ launch glue
template <int NP, bool GENERIC>
static cudaError_t launch_chunk_t(const ChunkArgs& a, int grid, size_t smem,
                                  cudaStream_t st) {
  auto fn = chunk_kernel<NP, GENERIC>;
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  return launch_cooperative(fn, grid, chunk_threads(GENERIC), smem, st, a);
}

template <int NP, bool GENERIC>
static int chunk_max_grid_t(size_t smem) {
  auto fn = chunk_kernel<NP, GENERIC>;
  if (allow_max_smem(fn) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, chunk_threads(GENERIC),
                                                    smem) != cudaSuccess)
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
    case 28: return launch_chunk_t<28, false>(a, grid, smem, st);
    default: return launch_chunk_t<32, false>(a, grid, smem, st);
  }
}

int chunk_max_grid(bool generic, int np, size_t smem) {
  if (generic) return chunk_max_grid_t<0, true>(smem);
  switch (np) {
    case 4: return chunk_max_grid_t<4, false>(smem);
    case 8: return chunk_max_grid_t<8, false>(smem);
    case 16: return chunk_max_grid_t<16, false>(smem);
    case 28: return chunk_max_grid_t<28, false>(smem);
    default: return chunk_max_grid_t<32, false>(smem);
  }
}

size_t assign_smem(int npad, int k, int kpad, bool generic) {
  if (!generic)
    return align_up(k * npad * 4, 16) + align_up(k * 4, 16) + align_up((k + 1) * 4, 16) + 64 * 8;
  return align_up(npad * kpad * 4, 16) + align_up(k * 4, 16) +
         align_up(64 * npad * 4, 16) + 64 * 8;
}

template <typename F>
static int max_grid_of(F fn, size_t smem) {
  if (allow_max_smem(fn) != cudaSuccess) return 0;
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
    case 28: return max_grid_of(assign_np_kernel<28>, smem);
    default: return max_grid_of(assign_np_kernel<32>, smem);
  }
}

cudaError_t launch_x_ready(uint32_t* landed, uint32_t count, cudaStream_t st) {
  x_ready_kernel<<<1, 1, 0, st>>>(landed, count);
  return cudaGetLastError();
}

cudaError_t launch_assign(const AssignArgs& a, int grid, bool generic, int np,
                          size_t smem, cudaStream_t st) {
  if (generic) {
    allow_max_smem(assign_generic_kernel);
    assign_generic_kernel<<<grid, kThreads, smem, st>>>(a);
  } else {
    switch (np) {
      case 4:
        allow_max_smem(assign_np_kernel<4>);
        assign_np_kernel<4><<<grid, kThreads, smem, st>>>(a);
        break;
      case 8:
        allow_max_smem(assign_np_kernel<8>);
        assign_np_kernel<8><<<grid, kThreads, smem, st>>>(a);
        break;
      case 16:
        allow_max_smem(assign_np_kernel<16>);
        assign_np_kernel<16><<<grid, kThreads, smem, st>>>(a);
        break;
      case 28:
        allow_max_smem(assign_np_kernel<28>);
        assign_np_kernel<28><<<grid, kThreads, smem, st>>>(a);
        break;
      default:
        allow_max_smem(assign_np_kernel<32>);
        assign_np_kernel<32><<<grid, kThreads, smem, st>>>(a);
        break;
    }
  }
  return cudaGetLastError();
}

}  // namespace bm
