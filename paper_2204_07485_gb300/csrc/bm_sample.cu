// Sample plan: the uniform samples of a batch of chunks, drawn in one launch.
//
// Alg. 1 draws a fresh uniform sample of s rows for every chunk (Sec. 3.1,
// Eq. 2; Sec. 3.5).  The draws do not depend on the incumbent, so a batch of
// B chunks is drawn ahead by one launch with one CTA per chunk, all chunks in
// parallel, off the per-chunk critical path.  Per chunk t:
//   round r draws (target - |S|) Philox words (purpose 0, counter
//   (i / 4, r, t, 0)), maps each to a row by the high word of w * m, and adds
//   it to S with atomicOr on the chunk's bitmap (in shared memory when it
//   fits); |S| grows by the count of atomics that found their bit clear.
//   Rounds continue until |S| = target (64 rounds at most; the smallest
//   absent rows complete S after that, which never happens in practice for
//   target <= m / 2).  target = s, or m - s rows to leave out when 2s > m.
//   A fixed-order scan of the bitmap then writes the sample's rows in
//   ascending order (and clears a global bitmap for the next use).
// Nothing here waits on another CTA.
#include <cuda_runtime.h>

#include "bm_device.cuh"
#include "bm_internal.h"

namespace bm {

constexpr int kDrawThreads = 512;
constexpr int kWordsPerThread = 8;

__device__ __forceinline__ int block_excl_scan_i32(int v, int* buf, int* total) {
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

// Bits of bitmap word w that mark sample rows: the word itself, or for a
// complement draw the rows left unmarked (within [0, m)).
__device__ __forceinline__ uint32_t sample_bits(uint32_t raw, long long w, long long W,
                                                long long m, bool complement) {
  if (!complement) return raw;
  if (w >= W) return 0u;
  uint32_t v = ~raw;
  const long long lo = w * 32;
  if (lo + 32 > m) v &= (1u << (m - lo)) - 1u;
  return v;
}

__global__ void __launch_bounds__(kDrawThreads) draw_kernel(DrawArgs a) {
  extern __shared__ __align__(16) uint32_t sbits[];   // the chunk's bitmap, when it fits
  BM_POISON_SMEM();
  __shared__ int red[32];
  __shared__ int scan[32];
  const long long W = (a.m + 31) / 32;
  const long long t = a.t0 + blockIdx.x;
  const bool in_smem = a.smem_bitmap != 0;
  uint32_t* bm = in_smem ? sbits : a.bitmaps + (size_t)blockIdx.x * draw_bitmap_words(a.m);
  int32_t* out = a.idx + (size_t)blockIdx.x * a.s;
  const bool complement = 2 * (long long)a.s > a.m;
  const uint32_t target = complement ? (uint32_t)(a.m - a.s) : (uint32_t)a.s;
  if (in_smem) {
    for (long long w = threadIdx.x; w < W; w += blockDim.x) sbits[w] = 0u;
    __syncthreads();
  }

  // Round r draws (target - |S|) values.  One Philox evaluation gives the
  // four words of counter c = i / 4, so a thread takes four consecutive
  // draws at a time.  |S| grows by the number of atomics that found their
  // bit clear: a value drawn several times flips its bit exactly once, so
  // the count does not depend on the order of the atomics.
  uint32_t have = 0;
  for (int r = 0; r < kRoundSlots && have < target; ++r) {
    const uint32_t need = target - have;
    const uint32_t blocks = (need + 3u) / 4u;
    int got = 0;
    for (uint32_t c = threadIdx.x; c < blocks; c += blockDim.x) {
      const U64x4 w4 = philox4x64_10(c, (uint64_t)r, (uint64_t)t, 0, a.seed, 0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (4u * c + (uint32_t)q < need) {
          const uint64_t v = __umul64hi(w4.x[q], (uint64_t)a.m);
          const uint32_t bit = 1u << (v & 31);
          if (!BM_GUARD(v < (uint64_t)a.m, a.status)) continue;
          const uint32_t old = atomicOr(bm + (v >> 5), bit);
          got += (old & bit) ? 0 : 1;
        }
      }
    }
    have += (uint32_t)block_sum_i32(got, red);
  }
  if (have < target && threadIdx.x == 0) {
    for (long long w = 0; w < W && have < target; ++w) {
      uint32_t word = in_smem ? bm[w] : __ldcg(bm + w);
      for (int bpos = 0; bpos < 32 && have < target; ++bpos) {
        if (w * 32 + bpos >= a.m) break;
        if (!(word & (1u << bpos))) { word |= 1u << bpos; ++have; }
      }
      bm[w] = word;
    }
  }
  __syncthreads();

  if (!in_smem) {
    // global bitmap: thread i owns the contiguous 16-byte groups [g0, g1);
    // a first pass counts its sample rows (eight loads in flight), an
    // exclusive scan gives its first output position, a second pass writes
    // its rows in ascending order and clears the words for the next draw
    const long long G4 = (long long)draw_bitmap_words(a.m) / 4;
    const long long span = (G4 + blockDim.x - 1) / blockDim.x;
    const long long g0 = min(G4, (long long)threadIdx.x * span), g1 = min(G4, g0 + span);
    uint4* b4 = reinterpret_cast<uint4*>(bm);
    int cnt = 0;
    for (long long g = g0; g < g1; g += 8) {
      uint4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = g + u < g1 ? __ldcg(b4 + g + u) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const long long w = 4 * (g + u);
        if (g + u < g1)
          cnt += __popc(sample_bits(v[u].x, w, W, a.m, complement)) +
                 __popc(sample_bits(v[u].y, w + 1, W, a.m, complement)) +
                 __popc(sample_bits(v[u].z, w + 2, W, a.m, complement)) +
                 __popc(sample_bits(v[u].w, w + 3, W, a.m, complement));
      }
    }
    int total;
    int pos = block_excl_scan_i32(cnt, scan, &total);
    for (long long g = g0; g < g1; g += 8) {
      uint4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = g + u < g1 ? __ldcg(b4 + g + u) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (g + u >= g1) continue;
        const uint32_t raw[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long w = 4 * (g + u) + e;
          uint32_t bits = sample_bits(raw[e], w, W, a.m, complement);
          while (bits) {
            const int bp = __ffs(bits) - 1;
            if (pos < a.s) out[pos] = (int32_t)(w * 32 + bp);
            ++pos;
            bits &= bits - 1;
          }
        }
        if (v[u].x | v[u].y | v[u].z | v[u].w) b4[g + u] = make_uint4(0, 0, 0, 0);
      }
    }
    return;
  }

  // shared-memory bitmap: kWordsPerThread consecutive words per thread per tile
  int base = 0;
  const long long tile = (long long)blockDim.x * kWordsPerThread;
  for (long long t0 = 0; t0 < W; t0 += tile) {
    const long long wb = t0 + (long long)threadIdx.x * kWordsPerThread;
    uint32_t words[kWordsPerThread];
    int c = 0;
#pragma unroll
    for (int u = 0; u < kWordsPerThread; ++u) {
      const long long w = wb + u;
      const uint32_t v = w < W ? sample_bits(bm[w], w, W, a.m, complement) : 0u;
      words[u] = v;
      c += __popc(v);
    }
    int total;
    int pos = base + block_excl_scan_i32(c, scan, &total);
#pragma unroll
    for (int u = 0; u < kWordsPerThread; ++u) {
      uint32_t bits = words[u];
      while (bits) {
        const int bp = __ffs(bits) - 1;
        if (pos < a.s) out[pos] = (int32_t)((wb + u) * 32 + bp);
        ++pos;
        bits &= bits - 1;
      }
    }
    base += total;
  }
}

// Bitmaps up to this size live in shared memory (m up to 1.6 million rows).
constexpr size_t kDrawSmemBitmap = 200 * 1024;

cudaError_t launch_draw(const DrawArgs& a, int chunks, cudaStream_t st) {
  DrawArgs d = a;
  const size_t bytes = (size_t)((a.m + 31) / 32) * 4;
  d.smem_bitmap = bytes <= kDrawSmemBitmap ? 1 : 0;
  if (d.smem_bitmap) {
    const cudaError_t e = allow_max_smem(draw_kernel);
    if (e != cudaSuccess) return e;
  }
  draw_kernel<<<chunks, kDrawThreads, d.smem_bitmap ? bytes : 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace bm
