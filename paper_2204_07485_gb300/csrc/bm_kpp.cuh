// K-means++ candidate selection shared by the chunk kernels (Sec. 3.3,
// three candidates per Sec. 5): the inverse-CDF search for each candidate's
// row over the per-CTA D^2 sums and, once the candidates' potentials are
// summed per CTA, the choice of the lowest potential.  Both run identically
// in every CTA, so every CTA reaches the same decision without a broadcast.
//
// Every value one CTA hands to the others here (its D^2 block sum, its
// candidates' potentials, a candidate row) is published with a tag: the
// value is stored, then a tag unique to (launch generation, slot j) is stored
// with release semantics, and a reader acquires the tag before it reads the
// value.  The grid barrier between writer and reader already orders them, so
// the first poll normally finds the tag; a reader that finds an older one
// counts a late read in Ctl::late and waits (bounded) for the right tag.  A
// value is therefore never used before it was written, whatever the barrier
// did, and any such event is visible to the host.
#pragma once

#include "bm_device.cuh"
#include "bm_internal.h"

namespace bm {

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Slots a warp reads per page of a per-CTA exchange: lane l holds slots
// l, l + 32, ... (kKxLanes of them), so one page costs one round trip.
constexpr int kKxLanes = 8;
constexpr int kKxPage = 32 * kKxLanes;

// Launch generation: read by every CTA at the start of a launch (the previous
// launch on the workspace has completed), advanced by CTA 0 at its end.
__device__ __forceinline__ unsigned long long kx_generation(const ChunkArgs& a) {
  return __ldcg(a.kx);
}
__device__ __forceinline__ void kx_advance(const ChunkArgs& a, unsigned long long gen) {
  a.kx[0] = gen + 1ull;
}
// Tag of slot j's exchange in launch generation gen (never 0: the tags start
// zeroed, so no stale tag equals a current one).
__device__ __forceinline__ unsigned long long kx_tag(unsigned long long gen, int j) {
  return (gen << 32) | (unsigned long long)(uint32_t)(j + 1);
}
__device__ __forceinline__ unsigned long long* kx_dsum(const ChunkArgs& a) { return a.kx + 1; }
__device__ __forceinline__ unsigned long long* kx_pot(const ChunkArgs& a) {
  return a.kx + 1 + gridDim.x;
}
__device__ __forceinline__ unsigned long long* kx_cand(const ChunkArgs& a) {
  return a.kx + 1 + 2 * gridDim.x;
}

// Waits until *tag == want.  Normally the first acquire succeeds.  Otherwise
// counts a late read and polls with the grid barrier's bounds; gives up with
// BM_ETIMEOUT in the status word (or when another CTA recorded an error) and
// returns false.
static __device__ __noinline__ bool kx_wait(const ChunkArgs& a, const unsigned long long* tag,
                                     unsigned long long want) {
  if (ld_acquire_u64(tag) == want) return true;
  atomicAdd(&a.ctl->late, 1u);
  uint64_t t0 = 0;
  uint32_t polls = 0;
  while (ld_acquire_u64(tag) != want) {
    ++polls;
    if ((polls & 255u) == 0) {
      const uint64_t now = global_timer_ns();
      if (t0 == 0) t0 = now;
      if (ld_volatile(&a.ctl->status) != kStatusOk || polls > kSpinLimit ||
          now - t0 > kSpinTimeoutNs) {
        atomicCAS(&a.ctl->status, kStatusOk, kStatusTimeout);
        return false;
      }
    }
    __nanosleep(32);
  }
  return true;
}

// The calling warp acquires tags[0, count) == want: a page's tags are read
// with relaxed loads, all in flight together; a tag that is not yet current
// is waited for (kx_wait); then one acquire fence orders every later read
// after all the tags.  Every lane gets true when all arrived.
__device__ __forceinline__ bool kx_wait_warp(const ChunkArgs& a, const unsigned long long* tags,
                                             int count, unsigned long long want) {
  const int l = threadIdx.x & 31;
  bool ok = true;
  for (int p0 = 0; p0 < count; p0 += kKxPage) {
    unsigned long long v[kKxLanes];
#pragma unroll
    for (int i = 0; i < kKxLanes; ++i) {
      const int x = p0 + l + 32 * i;
      v[i] = x < count ? ld_relaxed_u64(tags + x) : want;
    }
#pragma unroll
    for (int i = 0; i < kKxLanes; ++i)
      if (v[i] != want) ok = kx_wait(a, tags + p0 + l + 32 * i, want) && ok;
  }
  fence_acq_rel_gpu();
  return __all_sync(0xffffffffu, ok);
}

// Thread 0 publishes this CTA's D^2 block sum for slot j.
__device__ __forceinline__ void kpp_put_dsum(const ChunkArgs& a, double* DSUM, double v,
                                             unsigned long long tag) {
  if (threadIdx.x == 0) {
    DSUM[blockIdx.x] = v;
    st_release_u64(kx_dsum(a) + blockIdx.x, tag);
  }
}

// Thread 0 publishes this CTA's candidate potentials (part_f[t][b], t < trials).
__device__ __forceinline__ void kpp_put_potentials(const ChunkArgs& a, const double* v,
                                                   unsigned long long tag) {
  if (threadIdx.x == 0) {
    for (int t = 0; t < a.trials; ++t) a.part_f[(size_t)t * gridDim.x + blockIdx.x] = v[t];
    st_release_u64(kx_pot(a) + blockIdx.x, tag);
  }
}

__device__ __forceinline__ void kpp_put_cand(const ChunkArgs& a, int t, int row,
                                             unsigned long long tag) {
  a.ctl->cand[t] = row;
  st_release_u64(kx_cand(a) + t, tag);
}

// Candidate rows of slot j into rows[0..trials) (shared); every thread gets
// them.  Ends with a block barrier; false if a wait gave up.
__device__ __forceinline__ bool kpp_get_cands(const ChunkArgs& a, int* rows,
                                              unsigned long long tag) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  if (threadIdx.x < a.trials) {
    if (kx_wait(a, kx_cand(a) + threadIdx.x, tag)) rows[threadIdx.x] = __ldcg(a.ctl->cand + threadIdx.x);
    else s_ok = 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Targets u_t * sum(D^2) for the trials of slot j; the CTA holding target t
// (inclusive prefix over CTAs, then over its own rows in index order)
// publishes the row as candidate t.  A zero total falls back to a uniform row.
// DSUM[0..G) holds the CTAs' D^2 sums (published with tag); dmin[0..nrows)
// this CTA's D^2.  Returns false (every thread) if a wait gave up.
__device__ __forceinline__ bool kpp_locate(const ChunkArgs& a, const float* dmin, int r0,
                                           int nrows, const double* DSUM, int j,
                                           unsigned long long tag) {
  __shared__ double s_tgt[kMaxTrials], s_excl[kMaxTrials], s_total;
  __shared__ int s_bstar[kMaxTrials], s_ok;
  const int G = gridDim.x, b = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w == 0) {
    // every block sum's tag first: afterwards the sums are read as published
    const bool ok = kx_wait_warp(a, kx_dsum(a), G, tag);
    if (l == 0) s_ok = ok;
    // the sums of a page in registers (lane l: CTAs p0 + l + 32 i), all
    // loads in flight; the first page is kept for the prefix pass
    double first[kKxLanes];
    auto load_page = [&](int p0, double* dv) {
#pragma unroll
      for (int i = 0; i < kKxLanes; ++i) {
        const int x = p0 + l + 32 * i;
        dv[i] = x < G ? __ldcg(DSUM + x) : 0.0;
      }
    };
    double carry = 0.0;
    for (int p0 = 0; p0 < G; p0 += kKxPage) {
      double dv[kKxLanes];
      load_page(p0, dv);
#pragma unroll
      for (int i = 0; i < kKxLanes; ++i) {
        if (p0 == 0) first[i] = dv[i];
        if (p0 + 32 * i < G) carry += warp_sum_f64(dv[i]);
      }
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
      for (int p0 = 0; p0 < G; p0 += kKxPage) {
        double dv[kKxLanes];
        if (p0 == 0) {
#pragma unroll
          for (int i = 0; i < kKxLanes; ++i) dv[i] = first[i];
        } else {
          load_page(p0, dv);
        }
#pragma unroll
        for (int i = 0; i < kKxLanes; ++i) {
          const int base = p0 + 32 * i;
          if (base >= G) break;
          const double v = dv[i];
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
  if (!s_ok) return false;
  // the CTA that owns a target finds the row inside its block
  for (int t = 0; t < a.trials; ++t) {
    if (s_total == 0.0) {
      if (b == 0 && threadIdx.x == 0) {
        const double u = unit_double(philox_word(a.seed, (uint64_t)a.t, 2, 0,
                                                 (uint64_t)(j * a.trials + t)));
        kpp_put_cand(a, t, (int)floor(u * (double)a.s), tag);
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
      if (l == 0) kpp_put_cand(a, t, r0 + cand, tag);
    }
  }
  return true;
}

// Index of the trial with the lowest potential (sum over CTAs of
// part_f[t][u], fixed order, published with tag), lowest trial on ties; -1
// (every thread) if a wait gave up.  Ends with a block barrier.
__device__ __forceinline__ int kpp_best(const ChunkArgs& a, unsigned long long tag) {
  __shared__ int s_best;
  const int G = gridDim.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w == 0) {
    const bool ok = kx_wait_warp(a, kx_pot(a), G, tag);
    double v[kMaxTrials];
#pragma unroll
    for (int t = 0; t < kMaxTrials; ++t) v[t] = 0.0;
    // a page's potentials in registers first (all loads in flight), then
    // added per trial over u = l, l + 32, ... in order
    for (int p0 = 0; p0 < G; p0 += kKxPage) {
      double pv[kKxLanes][kMaxTrials];
#pragma unroll
      for (int i = 0; i < kKxLanes; ++i) {
        const int u = p0 + l + 32 * i;
#pragma unroll
        for (int t = 0; t < kMaxTrials; ++t)
          pv[i][t] = (u < G && t < a.trials) ? __ldcg(a.part_f + (size_t)t * G + u) : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kKxLanes; ++i)
#pragma unroll
        for (int t = 0; t < kMaxTrials; ++t)
          if (p0 + l + 32 * i < G && t < a.trials) v[t] += pv[i][t];
    }
    int best = 0;
    double bestv = 0.0;
#pragma unroll
    for (int t = 0; t < kMaxTrials; ++t) {
      if (t < a.trials) {
        const double phi = warp_sum_f64(v[t]);
        if (t == 0 || phi < bestv) { bestv = phi; best = t; }
      }
    }
    if (l == 0) s_best = ok ? best : -1;
  }
  __syncthreads();
  return s_best;
}

}  // namespace bm
