// FP32 distance building blocks shared by the tiled kernels: the squared
// difference accumulator, 64-row tiles staged transposed in shared memory and
// the nearest live centroid of a staged tile.
#pragma once

#include <climits>

#include "bm_device.cuh"

namespace bm {

__device__ __forceinline__ float sq(float e, float acc) { return fmaf(e, e, acc); }

// 64-row tiles are staged transposed, element (f, r) at f * 64 + (r ^ swz(f)).
// The XOR moves whole 4-row groups, so 4 consecutive rows stay one aligned
// float4, lanes walking rows hit 32 distinct banks, and threads walking
// features see at most a 4-way bank conflict.
__device__ __forceinline__ int swz(int f) { return (f & 7) << 2; }

// stage <- rows [0, rows) of src (row stride `stride`), zero elsewhere.
__device__ __forceinline__ void stage_tile(float* stage, const float* src, size_t stride,
                           int rows, int n, int npad, bool vec4, bool coherent) {
  if (vec4) {
    const int nq = npad / 4;
    for (int e = threadIdx.x; e < 64 * nq; e += blockDim.x) {
      const int r = e & 63, q = e >> 6;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows && 4 * q < n) {
        const float4* p = reinterpret_cast<const float4*>(src + (size_t)r * stride) + q;
        v = coherent ? __ldcg(p) : __ldg(p);
      }
      const int f = 4 * q;
      stage[f * 64 + (r ^ swz(f))] = v.x;
      stage[(f + 1) * 64 + (r ^ swz(f + 1))] = v.y;
      stage[(f + 2) * 64 + (r ^ swz(f + 2))] = v.z;
      stage[(f + 3) * 64 + (r ^ swz(f + 3))] = v.w;
    }
  } else {
    for (int e = threadIdx.x; e < 64 * npad; e += blockDim.x) {
      const int r = e & 63, f = e >> 6;
      float v = 0.f;
      if (r < rows && f < n) {
        const float* p = src + (size_t)r * stride + f;
        v = coherent ? __ldcg(p) : __ldg(p);
      }
      stage[f * 64 + (r ^ swz(f))] = v;
    }
  }
  __syncthreads();
}

// Nearest live centroid of the 64 staged rows (8 warps x 8 rows, one lane
// per centroid of each group of 32); lane r of warp w reports tile row
// 8w + r through (bj, bd) and returns true when that row exists.
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
  for (int f = 0; f < n; ++f) {
    const float* sp = stage + f * 64;
    const int sz = swz(f);
    const float4 pa = *reinterpret_cast<const float4*>(sp + ((w * 8) ^ sz));
    const float4 pb = *reinterpret_cast<const float4*>(sp + ((w * 8 + 4) ^ sz));
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

}  // namespace bm
