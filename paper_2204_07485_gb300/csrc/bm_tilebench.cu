// Distance-tile pipeline with its operands resident in shared memory: the
// measurement that separates the tensor-core tile design (tcgen05.mma into
// TMEM, then the candidate epilogue of the chunk and assignment kernels)
// from the data movement around it.
//
// One persistent CTA per SM holds a few 128-row A tiles (BF16, or split BF16
// hi + lo) and the centroid block B in shared memory, loaded once.  Thread 0
// issues the MMAs of step s (tile s mod tiles, all K blocks) into TMEM
// accumulator buffer s mod B (B buffers of N columns, as many as TMEM's 512
// columns hold, at most 8); epilogue warpgroup s mod 2 (warps 4..7 or 8..11,
// one TMEM lane quarter per warp) reads the approximate distances of step s
// -- the chunk kernel's two passes: the minimum of ||c_j||^2 - 2 x.c_j over
// the live columns, then the count of columns within a threshold of it --
// and frees the buffer.  The MMAs of the next B - 1 steps overlap the
// epilogues.  With the epilogue off the warpgroups only free the buffers,
// which times the MMAs alone.
//
// Operands are small integers (exact in BF16, dot products exact in FP32), so
// the checksum -- argmin + 1024 x tie count, summed over rows and steps -- can
// be recomputed on the host exactly.
#include <algorithm>
#include <climits>
#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_device.cuh"
#include "bm_internal.h"
#include "bm_tc.cuh"

namespace bm {

constexpr int kTbRows = 128;
constexpr int kTbThreads = 384;     // warp 0: TMEM + MMA issue; warps 4..11: two epilogue warpgroups
constexpr int kTbMaxTiles = 4;
constexpr int kTbMaxBufs = 8;

// Operand patterns (restated by the test): A element (tile, row, feature),
// B element (centroid, feature).
__host__ __device__ inline int tb_a(int tile, int r, int f) {
  return ((r * 7 + f * 3 + tile * 5) % 5) - 2;
}
__host__ __device__ inline int tb_b(int j, int f) { return ((j * 11 + f * 13) % 7) - 3; }

struct TbArgs {
  int n, k, N, planes, tiles, steps, epilogue, bufs, ncols;
  unsigned long long* checksum;
  int* status;
};

struct TbLayout {
  int a, b, cc, bars, holder, total;
};

__host__ __device__ inline TbLayout tb_layout(int n, int N, int planes, int tiles) {
  const int kb = n / 64;
  TbLayout L;
  int o = 0;
  L.a = o;      o += tiles * planes * kb * kTbRows * 128;
  L.b = o;      o += planes * kb * N * 128;
  L.cc = o;     o += align_up(N + 32, 32) * 4;
  L.bars = o;   o += 2 * kTbMaxBufs * 8;
  L.holder = o; o += 16;
  L.total = o + 1024;   // alignment slack of the dynamic base
  return L;
}

__device__ __forceinline__ void tb_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(mbar)) : "memory");
}

__global__ void __launch_bounds__(kTbThreads, 1) tile_bench_kernel(TbArgs a) {
  extern __shared__ __align__(1024) unsigned char tb_raw[];
  BM_POISON_SMEM();
  unsigned char* sm = tb_raw + ((1024u - (smem_u32(tb_raw) & 1023u)) & 1023u);
  const int n = a.n, k = a.k, N = a.N, P = a.planes, T = a.tiles, kb = n / 64;
  const TbLayout L = tb_layout(n, N, P, T);
  unsigned char* sA = sm + L.a;
  unsigned char* sB = sm + L.b;
  float* cc = reinterpret_cast<float*>(sm + L.cc);
  uint64_t* mma_done = reinterpret_cast<uint64_t*>(sm + L.bars);   // [bufs]
  uint64_t* tmem_free = mma_done + kTbMaxBufs;                      // [bufs]
  const int NB = a.bufs;
  uint32_t* holder = reinterpret_cast<uint32_t*>(sm + L.holder);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int planeA = kb * kTbRows * 128, planeB = kb * N * 128, tileA = P * planeA;

  // ---- operands: exact BF16 hi planes, zero lo planes
  for (int e = tid; e < T * kb * kTbRows * 64; e += kTbThreads) {
    const int t = e / (kb * kTbRows * 64), rem = e - t * (kb * kTbRows * 64);
    const int b = rem / (kTbRows * 64), r = (rem >> 6) & (kTbRows - 1), f = rem & 63;
    const int off = t * tileA + b * (kTbRows * 128) + sw128_offset(r, f);
    *reinterpret_cast<__nv_bfloat16*>(sA + off) = __float2bfloat16_rn((float)tb_a(t, r, b * 64 + f));
    if (P == 2) *reinterpret_cast<__nv_bfloat16*>(sA + planeA + off) = __float2bfloat16_rn(0.f);
  }
  for (int e = tid; e < kb * N * 64; e += kTbThreads) {
    const int b = e / (N * 64), j = (e >> 6) % N, f = e & 63;
    const float v = j < k ? (float)tb_b(j, b * 64 + f) : 0.f;
    const int off = b * (N * 128) + sw128_offset(j, f);
    *reinterpret_cast<__nv_bfloat16*>(sB + off) = __float2bfloat16_rn(v);
    if (P == 2) *reinterpret_cast<__nv_bfloat16*>(sB + planeB + off) = __float2bfloat16_rn(0.f);
  }
  for (int j = tid; j < align_up(N + 32, 32); j += kTbThreads) {
    float s = INFINITY;
    if (j < k) {
      s = 0.f;
      for (int f = 0; f < n; ++f) s += (float)(tb_b(j, f) * tb_b(j, f));
    }
    cc[j] = s;
  }
  if (tid == 0) {
    for (int i = 0; i < NB; ++i) {
      mbar_init(mma_done + i, 1);
      mbar_init(tmem_free + i, kTbRows);
    }
    mbar_init_fence();
  }
  const int ncols = a.ncols;
  if (warp == 0) tmem_alloc(holder, (uint32_t)ncols);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;
  bool ok = true;
  unsigned long long sum = 0ull;

  if (tid == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16_f32(kTbRows, N);
    const uint64_t db = sdesc_sw128(smem_u32(sB));
    const uint64_t alo = (uint64_t)(planeA >> 4), blo = (uint64_t)(planeB >> 4);
    for (int s = 0; s < a.steps && ok; ++s) {
      const int buf = s % NB;
      if (s >= NB && !mbar_wait(tmem_free + buf, (uint32_t)(((s / NB) - 1) & 1))) ok = false;
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(buf * N);
      const uint64_t da = sdesc_sw128(smem_u32(sA + (s % T) * tileA));
      for (int b = 0; b < kb; ++b)
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t oa = (uint64_t)((b * kTbRows * 128 + ks * 32) >> 4);
          const uint64_t ob = (uint64_t)((b * N * 128 + ks * 32) >> 4);
          tc_mma_bf16(d, da + oa, db + ob, idesc, (b > 0 || ks > 0) ? 1u : 0u);
          if (P == 2) {
            tc_mma_bf16(d, da + oa, db + blo + ob, idesc, 1u);
            tc_mma_bf16(d, da + alo + oa, db + ob, idesc, 1u);
          }
        }
      tc_commit(mma_done + buf);
    }
  } else if (warp >= 4) {
    // ---- epilogue warpgroups: warpgroup eg takes steps eg, eg + 2, ...; row
    // r = TMEM lane r
    const int q = warp & 3, eg = (warp >> 2) - 1;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    for (int s = eg; s < a.steps; s += 2) {
      const int buf = s % NB;
      // the warp leaves together (the TMEM loads below are warp-wide)
      if (!__all_sync(0xffffffffu, mbar_wait(mma_done + buf, (uint32_t)((s / NB) & 1)))) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (a.epilogue) {
        const uint32_t cols = lane_base + (uint32_t)(buf * N);
        float m1 = INFINITY;
        int j1 = INT_MAX;
        for (int c0 = 0; c0 < N; c0 += 32) {
          float acc[32];
          tmem_ld32(cols + (uint32_t)c0, acc);
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const float d = c0 + u < N ? fmaf(-2.f, acc[u], cc[c0 + u]) : INFINITY;
            if (d < m1) { m1 = d; j1 = c0 + u; }
          }
        }
        const float thr = m1 + 0.5f;
        int nc = 0;
        for (int c0 = 0; c0 < N; c0 += 32) {
          float acc[32];
          tmem_ld32(cols + (uint32_t)c0, acc);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            nc += (c0 + u < N && fmaf(-2.f, acc[u], cc[c0 + u]) <= thr) ? 1 : 0;
        }
        sum += (unsigned long long)j1 + 1024ull * (unsigned long long)nc;
      }
      tc_fence_before();
      tb_arrive(tmem_free + buf);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0 && sum) atomicAdd(a.checksum, sum);
  }
  if (!ok) atomicCAS(a.status, kStatusOk, kStatusTimeout);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)ncols);
}

}  // namespace bm

using namespace bm;

extern "C" bm_status bm_tile_bench(int32_t n, int32_t k, int32_t planes, int32_t steps,
                                   int32_t epilogue, double* ms_out, uint64_t* checksum_out,
                                   int32_t* grid_out, int32_t* tiles_out, void* stream) {
  if (n < 64 || n > 256 || n % 64 != 0 || k < 1 || k > kMaxK || (planes != 1 && planes != 2) ||
      steps < 1)
    return BM_EINVAL;
  const int N = align_up(k, 16);
  const size_t limit = 227 * 1024 - 1024;
  int tiles = 0;
  for (int t = kTbMaxTiles; t >= 1; --t)
    if ((size_t)tb_layout(n, N, planes, t).total <= limit) { tiles = t; break; }
  if (tiles == 0) return BM_EUNSUPPORTED;
  const size_t smem = (size_t)tb_layout(n, N, planes, tiles).total;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BM_ECUDA;
  if (cudaFuncSetAttribute(tile_bench_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return BM_ECUDA;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 16) != cudaSuccess) return BM_ENOMEM;
  unsigned long long* cks = static_cast<unsigned long long*>(buf);
  int* status = reinterpret_cast<int*>(cks + 1);
  bm_status rc = BM_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // accumulator buffers: as many N-column buffers as 512 TMEM columns hold
  // (at most 8, at least 2) when the epilogue's 32-column loads of the last
  // buffer stay inside the allocation, a power of two of at least 32 columns
  int bufs = kTbMaxBufs;
  while (bufs > 2 && (bufs - 1) * N + align_up(N, 32) > 512) --bufs;
  int ncols = 32;
  while (ncols < (bufs - 1) * N + align_up(N, 32)) ncols <<= 1;
  TbArgs a{};
  a.n = n; a.k = k; a.N = N; a.planes = planes; a.tiles = tiles; a.steps = steps;
  a.bufs = bufs; a.ncols = ncols;
  a.epilogue = epilogue != 0; a.checksum = cks; a.status = status;
  if (cudaMemsetAsync(buf, 0, 16, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = BM_ECUDA;
  if (rc == BM_OK) {
    cudaEventRecord(e0, st);
    tile_bench_kernel<<<sms, kTbThreads, smem, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) rc = BM_ECUDA;
    cudaEventRecord(e1, st);
  }
  unsigned long long h = 0;
  int hs = 0;
  if (rc == BM_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                      cudaMemcpy(&h, cks, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
                      cudaMemcpy(&hs, status, 4, cudaMemcpyDeviceToHost) != cudaSuccess))
    rc = BM_ECUDA;
  float ms = 0.f;
  if (rc == BM_OK) cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc != BM_OK) return rc;
  if (hs != 0) return (bm_status)hs;
  if (ms_out) *ms_out = ms;
  if (checksum_out) *checksum_out = h;
  if (grid_out) *grid_out = sms;
  if (tiles_out) *tiles_out = tiles;
  return BM_OK;
}
