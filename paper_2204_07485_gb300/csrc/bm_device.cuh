// Device-side building blocks shared by the Big-means kernels: the Philox
// stream, bounded-wait grid barrier, deterministic reductions and the
// fixed-order argmin.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bm {

constexpr int kThreads = 256;            // threads per CTA (assign kernels, tiled chunk kernel)
constexpr int kWideThreads = 512;        // threads per CTA of the row-in-register chunk kernel
constexpr int kMaxRounds = 64;           // sample-draw rounds (never reached)

// Status codes written to the device status word (same values as bm_status).
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 4;
constexpr int kStatusGuard = 8;

// Index guards of the debug build (compiled with BM_DEBUG_GUARDS): a guarded
// access whose index falls outside its buffer is skipped and records
// kStatusGuard in the status word (when the kernel has one); nothing traps.
// Release builds compile every guard to `true`.
#ifdef BM_DEBUG_GUARDS
__device__ __forceinline__ bool guard_ok(bool in_bounds, int* status) {
  if (!in_bounds && status) atomicCAS(status, kStatusOk, kStatusGuard);
  return in_bounds;
}
#define BM_GUARD(cond, status) (::bm::guard_ok((cond), (status)))
#else
#define BM_GUARD(cond, status) (true)
#endif

// Checking builds (BM_DEBUG_GUARDS) also fill a kernel's dynamic shared
// memory with 0xFF bytes before it starts -- a NaN in FP32, BF16 and E4M3,
// -1 as an integer -- so that a read of a location the kernel never wrote
// changes its results instead of picking up an earlier kernel's leftovers.
// Called by every thread at the top of the kernel; release builds compile
// it to nothing.
#ifdef BM_DEBUG_GUARDS
__device__ __forceinline__ void poison_dynamic_smem() {
  extern __shared__ __align__(16) uint32_t bm_poison_base[];
  uint32_t bytes;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(bytes));
  for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) bm_poison_base[i] = 0xFFFFFFFFu;
  __syncthreads();
}
#define BM_POISON_SMEM() (::bm::poison_dynamic_smem())
#else
#define BM_POISON_SMEM() ((void)0)
#endif

// Bounds of every device-side spin: the wait gives up after this many polls
// or this much wall time (read from %globaltimer), whichever comes first.
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint64_t kSpinTimeoutNs = 2000000000ull;   // 2 s

// ------------------------------------------------------------ Philox4x64-10
// Salmon, Moraes, Dror, Shaw, SC'11: 10 rounds of two 64x64->128 products
// with multipliers M0, M1 and a Weyl key schedule W0, W1.
struct U64x4 { uint64_t x[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1,
                                               uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  return U64x4{{c0, c1, c2, c3}};
}

// Word i of stream (seed, chunk t, purpose, round): counter (i/4, round, t,
// purpose), key (seed, 0), output word i % 4.
__device__ __forceinline__ uint64_t philox_word(uint64_t seed, uint64_t t,
                                                uint64_t purpose, uint64_t rnd,
                                                uint64_t i) {
  U64x4 w = philox4x64_10(i >> 2, rnd, t, purpose, seed, 0);
  const int q = int(i & 3);
  return q == 0 ? w.x[0] : q == 1 ? w.x[1] : q == 2 ? w.x[2] : w.x[3];
}

// Top 53 bits scaled by 2^-53: a double in [0, 1), exact.
__device__ __forceinline__ double unit_double(uint64_t w) {
  return double(w >> 11) * 0x1.0p-53;
}

// ------------------------------------------------------------ memory helpers
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_volatile(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Checking builds (BM_DEBUG_GUARDS) also spread the starts of the CTAs of a
// cooperative launch: CTA b first spins (b mod 32) x 1,500 SM cycles (about
// 0.8 us per step at the boost clock, at most about 25 us; far inside the
// grid barrier's timeout).  A CTA's start then falls at many points of the
// first microseconds of CTA 0's work, so anything one CTA writes to global
// memory before the launch's first grid barrier while another reads it at
// its start shows up as a changed result, not as a rare wrong one.  Release
// builds compile it to nothing.
#ifdef BM_DEBUG_GUARDS
__device__ __forceinline__ void start_skew() {
  if (threadIdx.x == 0) {
    const long long wait = 1500ll * (long long)(blockIdx.x % 32u);
    const long long c0 = clock64();
    while (clock64() - c0 < wait) {
    }
  }
  __syncthreads();
}
#define BM_START_SKEW() (::bm::start_skew())
#else
#define BM_START_SKEW() ((void)0)
#endif

// ------------------------------------------------------------ grid barrier
// Monotone-counter barrier for a cooperative launch (all CTAs co-resident).
// Barrier number e completes when the counter reaches e * gridDim.x.  On
// GB300 it costs about 1.3 us at 152 CTAs (measured with a barrier-only
// kernel).  The waiting thread gives up after kSpinLimit polls or
// kSpinTimeoutNs, or as soon as another CTA has recorded an error, records
// BM_ETIMEOUT and returns false; callers then leave the kernel.
struct GridBarrier {
  uint32_t* counter;
  int* status;
  uint32_t epoch;
  uint32_t expected = 0;                  // arrivals per barrier (0: every CTA of the grid)
  uint64_t timeout_ns = kSpinTimeoutNs;

  __device__ bool sync() {
    __shared__ int s_ok;
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
      const uint32_t target = epoch * (expected ? expected : gridDim.x);
      __threadfence();
      atomicAdd(counter, 1u);
      int ok = 1;
      uint64_t t0 = 0;   // read lazily: a fast barrier reads no timer
      uint32_t polls = 0;
      while (ld_acquire(counter) < target) {
        ++polls;
        if ((polls & 255u) == 0) {
          const uint64_t now = global_timer_ns();
          if (t0 == 0) t0 = now;
          if (ld_volatile(status) != kStatusOk || polls > kSpinLimit ||
              now - t0 > timeout_ns) {
            atomicCAS(status, kStatusOk, kStatusTimeout);
            ok = 0;
            break;
          }
        }
        __nanosleep(20);
      }
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  }
};

// ------------------------------------------------------------ reductions
// Fixed-order sums: the result depends only on the inputs and blockDim, so
// every CTA computing the same sum gets the same bits.
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_sum_i32(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide fixed-order FP64 sum; every thread gets the result.  red holds
// one slot per warp plus one (at most 33).  FP64 arithmetic is slow on this
// part, so only thread 0 adds up the per-warp sums.
__device__ __forceinline__ double block_sum_f64(double v, double* red) {
  v = warp_sum_f64(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}
__device__ __forceinline__ int block_sum_i32(int v, int* red) {
  v = warp_sum_i32(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  int t = 0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// Error-free FP32 accumulation (TwoSum): (hi, lo) += x, where lo collects the
// exact rounding error of every addition into hi.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// Fixed-order warp reduction of (hi, lo) pairs with TwoSum at every level,
// so hi + lo carries the sum of the 32 inputs to about 2^-48 relative.  The
// tree is symmetric in the two partners, so every lane ends with the same
// pair.  Used instead of FP64 shuffles: FP64 arithmetic is slow on this part.
__device__ __forceinline__ void warp_two_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, ohi);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(ohi, bb));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, olo), err);
  }
}

// Sum of x[0..len) (L2-coherent loads) by one warp in a fixed order; every
// lane gets the result.
// Lane l's sum of x[l], x[l + 32], x[l + 64], ... (in that order) from L2;
// the loads of up to eight terms go out together, so a grid's worth of
// partials (up to 256 CTAs) costs one round trip.  Absent terms add +0.
template <typename T>
__device__ __forceinline__ T lane_sum_ldcg(const T* x, int len) {
  const int l = threadIdx.x & 31;
  T v = T(0);
  for (int i0 = 0; i0 < len; i0 += 256) {
    T t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + 32 * u + l;
      t[u] = i < len ? __ldcg(x + i) : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) v += t[u];
  }
  return v;
}

__device__ __forceinline__ double warp_sum_array_f64(const double* x, int len) {
  return warp_sum_f64(lane_sum_ldcg(x, len));
}

// (d, j) argmin with the lowest index winning ties.
__device__ __forceinline__ bool better(float d, int j, float bd, int bj) {
  return d < bd || (d == bd && j < bj);
}
__device__ __forceinline__ void warp_argmin(float& d, int& j) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float od = __shfl_xor_sync(0xffffffffu, d, o);
    const int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (better(od, oj, d, j)) { d = od; j = oj; }
  }
}

}  // namespace bm
