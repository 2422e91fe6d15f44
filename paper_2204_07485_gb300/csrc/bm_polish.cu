// Full-data Lloyd polish (the extra SSE gain the paper suggests after
// Big-means, Sec. 3.4): Lloyd iterations (Sec. 2, stop rule of Sec. 5) on all
// of X from the incumbent.  The assignment pass is the final-assignment
// kernel; this file holds the update: per-CTA sums of (x - c_label) and
// member counts over a fixed contiguous range of rows, then a fixed-order sum
// over CTAs and the new centroids.  Every sum has a fixed order, so results
// are reproducible.
#include <cuda_runtime.h>

#include "bm_device.cuh"
#include "bm_internal.h"

namespace bm {

constexpr int kPolishThreads = 256;
constexpr int kPolishFpl = 8;    // features per lane: blocks of at most 256 features

// Features [f0, f0 + fw) of the update: warp w of a CTA adds its rows
// r0 + w, r0 + w + wu, ... in row order into a private slice acc[w][k][fw]
// (lane = feature), then the slices are added in warp order into this CTA's
// partials.  Warps >= wu only help with the set-up and the combination.
__global__ void __launch_bounds__(kPolishThreads) polish_accum_kernel(PolishArgs a) {
  extern __shared__ __align__(16) float psm[];
  BM_POISON_SMEM();
  const int k = a.k, npad = a.npad, wu = a.wu, f0 = a.f0, fw = a.fw;
  const int n = min(a.n - f0, fw);                   // features of this block
  float* cen = psm;                                  // [k][fw] current centroids
  float* acc = cen + (size_t)k * fw;                 // [wu][k][fw]
  int* cnt = reinterpret_cast<int*>(acc + (size_t)wu * k * fw);   // [wu][k]
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int q = threadIdx.x; q < k * fw; q += blockDim.x) {
    const int j = q / fw, f = q - j * fw;
    cen[q] = f < n ? __ldg(a.C + (size_t)j * a.cstride + f0 + f) : 0.f;
  }
  for (int q = threadIdx.x; q < wu * k * fw; q += blockDim.x) acc[q] = 0.f;
  for (int q = threadIdx.x; q < wu * k; q += blockDim.x) cnt[q] = 0;
  __syncthreads();
  const long long r0 = (long long)blockIdx.x * a.rows_per_cta;
  const long long r1 = min(a.m, r0 + a.rows_per_cta);
  if (w < wu) {
    float* my = acc + (size_t)w * k * fw;
    int* myc = cnt + w * k;
    // four rows per step: their loads go out together, their additions
    // follow in row order
    for (long long rb = r0 + w; rb < r1; rb += 4LL * wu) {
      int jj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long r = rb + (long long)u * wu;
        jj[u] = r < r1 ? __ldg(a.labels + r) : -1;
        if (jj[u] >= k) jj[u] = -1;
      }
      float xv[4][kPolishFpl];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float* x = a.X + (size_t)(rb + (long long)u * wu) * a.n + f0;
#pragma unroll
        for (int q = 0; q < kPolishFpl; ++q) {
          const int f = l + 32 * q;
          xv[u][q] = (jj[u] >= 0 && f < n) ? __ldg(x + f) : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = jj[u];
        if (j < 0) continue;
#pragma unroll
        for (int q = 0; q < kPolishFpl; ++q) {
          const int f = l + 32 * q;
          if (f < n) my[j * fw + f] += xv[u][q] - cen[j * fw + f];
        }
        if (l == 0) myc[j] += 1;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  float* ps = a.part_sum + (size_t)blockIdx.x * k * npad;
  for (int q = threadIdx.x; q < k * fw; q += blockDim.x) {
    const int j = q / fw, f = q - j * fw;
    if (f0 + f >= npad) continue;
    float s = 0.f;
    for (int u = 0; u < wu; ++u) s += acc[(size_t)u * k * fw + q];
    ps[(size_t)j * npad + f0 + f] = s;
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    int c = 0;
    for (int u = 0; u < wu; ++u) c += cnt[u * k + j];
    a.part_cnt[(size_t)blockIdx.x * k + j] = c;
  }
}

// New centroids: thread per (j, f); CTA partials added in CTA order, sixteen
// loads in flight.  A live centroid without members becomes degenerate
// (Sec. 3.3) whether or not the iteration stops, or with empty_keep stays
// where it is; the others move to c + sum / count unless it stops.
__global__ void __launch_bounds__(kPolishThreads) polish_reduce_kernel(PolishArgs a, int G,
                                                                      int stop) {
  const int k = a.k, npad = a.npad, n = a.n;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * npad) return;
  const int j = q / npad, f = q - j * npad;
  if (!a.mask[j]) return;
  int cnt = 0;
  float sum = 0.f;
  for (int b0 = 0; b0 < G; b0 += 16) {
    int cv[16];
    float sv[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int b = b0 + e;
      cv[e] = b < G ? __ldcg(a.part_cnt + (size_t)b * k + j) : 0;
      sv[e] = b < G ? __ldcg(a.part_sum + ((size_t)b * k + j) * npad + f) : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      cnt += cv[e];
      sum += sv[e];
    }
  }
  if (cnt == 0) {   // every thread of centroid j sees the same count
    if (!a.empty_keep && f == 0) a.mask[j] = 0;
    return;
  }
  if (!stop && f < n) {
    float* c = a.C + (size_t)j * a.cstride + f;
    *c = *c + sum / (float)cnt;
  }
}

size_t polish_smem(int k, int fw, int wu) {
  return (size_t)k * fw * 4 + (size_t)wu * k * fw * 4 + (size_t)wu * k * 4;
}

cudaError_t launch_polish_update(const PolishArgs& a, int grid, size_t smem, int stop,
                                 cudaStream_t st) {
  cudaError_t e = allow_max_smem(polish_accum_kernel);
  if (e != cudaSuccess) return e;
  for (int f0 = 0; f0 < a.n; f0 += a.fw) {   // one pass over X per feature block
    PolishArgs b = a;
    b.f0 = f0;
    polish_accum_kernel<<<grid, kPolishThreads, smem, st>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int kn = a.k * a.npad;
  polish_reduce_kernel<<<(kn + kPolishThreads - 1) / kPolishThreads, kPolishThreads, 0, st>>>(
      a, grid, stop);
  return cudaGetLastError();
}

}  // namespace bm
