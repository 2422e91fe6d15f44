// K-means++ candidate selection shared by the chunk kernels (Sec. 3.3,
// three candidates per Sec. 5): the inverse-CDF search for each candidate's
// row over the per-CTA D^2 sums and, once the candidates' potentials are
// summed per CTA, the choice of the lowest potential.  Both run identically
// in every CTA, so every CTA reaches the same decision without a broadcast.
#pragma once

#include "bm_device.cuh"
#include "bm_internal.h"

namespace bm {

// Targets u_t * sum(D^2) for the trials of slot j; the CTA holding target t
// (inclusive prefix over CTAs, then over its own rows in index order) writes
// the row into ctl->cand[t].  A zero total falls back to a uniform row.
// DSUM[0..G) holds the CTAs' D^2 sums; dmin[0..nrows) this CTA's D^2.
// The caller's next grid barrier publishes ctl->cand.
__device__ __forceinline__ void kpp_locate(const ChunkArgs& a, const float* dmin, int r0,
                                           int nrows, const double* DSUM, int j) {
  __shared__ double s_tgt[kMaxTrials], s_excl[kMaxTrials], s_total;
  __shared__ int s_bstar[kMaxTrials];
  const int G = gridDim.x, b = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
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
        const double v = base + l < nrows ? (double)dmin[base + l] : 0.0;
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
}

// Index of the trial with the lowest potential (sum over CTAs of
// part_f[t][u], fixed order), lowest trial on ties.  Ends with a block barrier.
__device__ __forceinline__ int kpp_best(const ChunkArgs& a) {
  __shared__ int s_best;
  const int G = gridDim.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w == 0) {
    double v[kMaxTrials];
#pragma unroll
    for (int t = 0; t < kMaxTrials; ++t) v[t] = 0.0;
    for (int u = l; u < G; u += 32)
#pragma unroll
      for (int t = 0; t < kMaxTrials; ++t)
        if (t < a.trials) v[t] += __ldcg(a.part_f + (size_t)t * G + u);
    int best = 0;
    double bestv = 0.0;
#pragma unroll
    for (int t = 0; t < kMaxTrials; ++t) {
      if (t < a.trials) {
        const double phi = warp_sum_f64(v[t]);
        if (t == 0 || phi < bestv) { bestv = phi; best = t; }
      }
    }
    if (l == 0) s_best = best;
  }
  __syncthreads();
  return s_best;
}

}  // namespace bm
