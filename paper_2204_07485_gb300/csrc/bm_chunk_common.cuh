// Pieces shared by the chunk kernels: CTA 0's phase timers, the live
// centroid list and the fixed-order sum of per-row minima.
#pragma once

#include "bm_device.cuh"
#include "bm_internal.h"

namespace bm {

// Phase timers of CTA 0, accumulated in shared memory during the launch and
// added to Stats::phase_ns once at its end (a global read-modify-write per
// tick would stall CTA 0, and through the next grid barrier every CTA).
__device__ __forceinline__ unsigned long long* phase_slots() {
  __shared__ unsigned long long slots[kNumPhaseTimers];
  return slots;
}

// Tracing is off unless the launch asks for it: a timer read on CTA 0's
// critical path delays every CTA at the next grid barrier.
__device__ __forceinline__ uint64_t trace_now(const ChunkArgs& a) {
  return a.trace ? global_timer_ns() : 0ull;
}

// Thread 0 of CTA 0 adds the time since *t0 to slot i (traced launches).
__device__ __forceinline__ void phase_tick(const ChunkArgs& a, int i, uint64_t* t0) {
  if (a.trace && blockIdx.x == 0 && threadIdx.x == 0) {
    const uint64_t t = global_timer_ns();
    phase_slots()[i] += t - *t0;
    *t0 = t;
  }
}

// Where a CTA gathers its sample rows from: X, or -- while X is still being
// filled by a copy from host memory in interleaved pieces (blocks of
// 2^x_shift rows, block b in piece b mod kHostCopyPieces, pieces landing in
// order) -- the host copy for the rows whose piece has not landed yet, read
// over the CPU-GPU link.  Both hold the same bytes, so the results do not
// depend on the choice.  gather_rows_ready returns the count of landed pieces
// for the whole gather (all of them without a host copy) and counts the
// gathers made before the last piece landed; called by all threads.
__device__ __forceinline__ long long gather_rows_ready(const ChunkArgs& a, int r0, int nrows) {
  (void)r0;
  if (!a.Xh) return kHostCopyPieces;
  __shared__ long long s_ready;
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long ready = (long long)ld_acquire(a.x_ready);
    s_ready = ready;
    if (nrows > 0 && ready < kHostCopyPieces)
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats->host_gathers), 1ull);
  }
  __syncthreads();
  return s_ready;
}
__device__ __forceinline__ const float* gather_row_source(const ChunkArgs& a, long long row,
                                                          long long ready) {
  if (!a.Xh) return a.X;
  return ((row >> a.x_shift) & (kHostCopyPieces - 1)) < ready ? a.X : a.Xh;
}
// Both sources allow 16-byte loads of rows whose length is a multiple of 4.
__device__ __forceinline__ bool gather_sources_aligned16(const ChunkArgs& a) {
  return (reinterpret_cast<uintptr_t>(a.X) & 15) == 0 &&
         (!a.Xh || (reinterpret_cast<uintptr_t>(a.Xh) & 15) == 0);
}

// lidx[0..c) <- indices of the live centroids in ascending order, lidx[k] = c.
// Called by all threads; ends with a barrier.
__device__ __forceinline__ void build_live_list(const int* live, int* lidx, int k) {
  __syncthreads();
  if (threadIdx.x < 32) {
    int c = 0;
    for (int base = 0; base < k; base += 32) {
      const int j = base + (int)threadIdx.x;
      const bool on = j < k && live[j];
      const unsigned bal = __ballot_sync(0xffffffffu, on);
      if (on) lidx[c + __popc(bal & ((1u << threadIdx.x) - 1u))] = j;
      c += __popc(bal);
    }
    if (threadIdx.x == 0) lidx[k] = c;
  }
  __syncthreads();
}

// Fixed-order sum of dmin[0..nrows), carried exactly in FP32 pairs (TwoSum)
// within each warp and added up in FP64 by one thread; every thread gets the
// result.  red holds at least 33 doubles.
__device__ __forceinline__ double dmin_sum(const float* dmin, int nrows, double* red) {
  float hi = 0.f, lo = 0.f;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) two_sum_acc(hi, lo, dmin[i]);
  warp_two_sum(hi, lo);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = (double)hi + (double)lo;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}

}  // namespace bm
