// Tensor-core nearest-centroid assignment (Alg. 1's final step, Sec. 3.4) in
// BF16 with exact FP32 rescoring.
//
// Distances are d_j = ||x||^2 - 2 x.c_j + ||c_j||^2 (Eq. 1 expanded); the
// dot products x.c_j of a 128-row tile against all k centroids run on the
// 5th-generation tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
// accumulators in TMEM).  BF16 rounding makes those distances approximate,
// so the epilogue bounds the error of every one of them,
//   |err_j| <= E_j = 2 eps ||x|| ||c_j|| + (n+2) 2^-22 ||c_j||^2
//                    + (n+4) 2^-22 (||x|| + ||c_j||)^2,
// with eps = 1.01 * 2^-7 + (n + 16) 2^-22 (two BF16 roundings of the
// operands plus FP32 accumulation), and keeps as candidates every centroid j
// with d_j - E_j <= min_i (d_i + E_i).  The candidate set provably contains
// the centroid that the exact FP32 distance picks; the candidates' exact FP32
// distances (four partial sums over f mod 4, the same arithmetic as the FP32
// kernels) then choose the label, lowest index on ties, and give the row's
// distance.  Labels and distances are therefore those of the FP32 path; only
// rows with more than one candidate ("rescored") pay for extra exact
// distances.
//
// The E4M3 form (FP8, single term) scales each row and each centroid by a
// power of two that brings its largest magnitude into [128, 256), so no
// operand saturates; the accumulator is scaled back exactly in the
// epilogue.  Each operand then carries a relative rounding error of at most
// 2^-4 plus an absolute error of 2^-10 / scale (the subnormal spacing), so
// eps = 2^-3 + 2^-8 + 2^-16 sqrt(n) + (n + 16) 2^-22 bounds the dot
// product's error relative to ||x|| ||c_j||; the candidate rule and the exact
// rescoring are those below.  Rows are converted a warp per row (every lane
// holds part of the row, so the row's maximum is a warp reduction).
//
// Data movement: each lane turns 8 consecutive FP32 features of a row into
// one 16-byte chunk of the 128-byte-swizzled BF16 K-major tile the MMA
// reads (and, in the split form, a second chunk with the low parts); row
// norms come from a shuffle over a row's chunks.  The centroid operand is
// built once per CTA.  Several CTAs share an SM (about 40-100 KB of shared
// memory each), so one CTA's loads overlap another's MMA and epilogue.
#include <algorithm>
#include <climits>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "bm_device.cuh"
#include "bm_internal.h"
#include "bm_tc.cuh"

// Compile-time tracing hook: BM_TC_TICK(i) marks the end of phase i of a
// tile (0 conversion, 1 MMA wait, 2 candidate scan, 3 rescoring, 4 barrier).
// It expands to nothing unless a profiling build defines it.
#ifndef BM_TC_TICK
#define BM_TC_TICK(i) ((void)0)
#endif

namespace bm {

constexpr int kTcRows = 128;       // MMA M: rows per tile, one thread per row
constexpr int kTcThreads = 128;

struct TcLayout {
  int sB, sA, stg, xF, cF, cc, xx, sc, red, bars, holder, total;
};

// planes = 1 (BF16) or 2 (hi and lo BF16 parts of the split form); stages:
// FP32 row tiles that bulk copies fill ahead (0: rows are loaded by the
// threads, with an FP32 copy for the exact distances when n <= 64); cF (FP32
// centroids for the exact distances) only when it fits.
__host__ __device__ inline TcLayout tc_layout(int n, int kb, int npad16, int k, int planes,
                                              bool cf, int stages) {
  TcLayout L;
  int o = 0;
  L.sB = o;    o += planes * kb * npad16 * 128;         // centroids, BF16 swizzled
  L.sA = o;    o += planes * kb * kTcRows * 128;        // row tile, BF16 swizzled
  L.stg = o;   o += stages * kTcRows * n * 4;           // FP32 row tiles (bulk copies)
  L.xF = o;    o += (stages == 0 && n <= 64) ? kTcRows * align_up(n, 4) * 4 : 0;
  L.cF = o;    o += cf ? align_up(k * n * 4, 16) : 0;   // FP32 centroids
  L.cc = o;    o += align_up(npad16 * 4, 16);           // ||c_j||^2, +inf if not live
  L.xx = o;    o += 2 * kTcRows * 4;                    // ||x||^2 of the tile's rows (two halves)
  L.sc = o;    o += (kTcRows + 128) * 4;                // E4M3 form: 1/scale of rows, centroids
  L.red = o;   o += 40 * 8;
  L.bars = o;  o += 8 * 3;                              // MMA completion, stage arrivals
  L.holder = o; o += 16;
  L.total = o;
  return L;
}

// Exact FP32 distance of row x and centroid c (either memory space): four
// partial sums over f mod 4, combined as (s0 + s1) + (s2 + s3) -- the same
// arithmetic as the FP32 kernels, so the results agree bit for bit.
__device__ __forceinline__ float dist_exact(const float* x, const float* c, int n, bool vec) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int f = 0;
  if (vec) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* c4 = reinterpret_cast<const float4*>(c);
#pragma unroll 8
    for (int q = 0; q < n / 4; ++q) {
      const float4 a = x4[q], b = c4[q];
      const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
      s0 = fmaf(e0, e0, s0);
      s1 = fmaf(e1, e1, s1);
      s2 = fmaf(e2, e2, s2);
      s3 = fmaf(e3, e3, s3);
    }
    return (s0 + s1) + (s2 + s3);
  }
  for (; f + 4 <= n; f += 4) {
    const float e0 = x[f] - c[f], e1 = x[f + 1] - c[f + 1];
    const float e2 = x[f + 2] - c[f + 2], e3 = x[f + 3] - c[f + 3];
    s0 = fmaf(e0, e0, s0);
    s1 = fmaf(e1, e1, s1);
    s2 = fmaf(e2, e2, s2);
    s3 = fmaf(e3, e3, s3);
  }
  if (f < n) { const float e = x[f] - c[f]; s0 = fmaf(e, e, s0); }
  if (f + 1 < n) { const float e = x[f + 1] - c[f + 1]; s1 = fmaf(e, e, s1); }
  if (f + 2 < n) { const float e = x[f + 2] - c[f + 2]; s2 = fmaf(e, e, s2); }
  return (s0 + s1) + (s2 + s3);
}

template <bool FP8>
__global__ void __launch_bounds__(kTcThreads, 4)
assign_tc_kernel(AssignTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw_tc[];
  BM_POISON_SMEM();
  // the swizzled tiles need a 1024-byte aligned base (the launch adds slack)
  unsigned char* smem_tc =
      smem_raw_tc + ((1024u - (smem_u32(smem_raw_tc) & 1023u)) & 1023u);
  const int n = a.n, k = a.k, kb = a.kb, N = a.npad16;
  const int planes = (!FP8 && a.terms == 3) ? 2 : 1;
  const bool cf = a.cf != 0;
  const int S = a.stages;   // FP32 row tiles in flight (0: thread loads)
  const TcLayout L = tc_layout(n, kb, N, k, planes, cf, S);
  unsigned char* sB = smem_tc + L.sB;
  unsigned char* sA = smem_tc + L.sA;
  float* cF = reinterpret_cast<float*>(smem_tc + L.cF);
  // the FP32 rows of the tile for the exact distances (rows padded to 4)
  const bool xf = S == 0 && n <= 64;
  float* stg = reinterpret_cast<float*>(smem_tc + L.stg);
  uint64_t* sbar = reinterpret_cast<uint64_t*>(smem_tc + L.bars) + 1;
  const int xs = align_up(n, 4);
  float* xF = reinterpret_cast<float*>(smem_tc + L.xF);
  float* cc = reinterpret_cast<float*>(smem_tc + L.cc);
  float* xx = reinterpret_cast<float*>(smem_tc + L.xx);
  float* rsc = reinterpret_cast<float*>(smem_tc + L.sc);   // E4M3: 1 / row scale
  float* csc = rsc + kTcRows;                               // E4M3: 1 / centroid scale
  double* red = reinterpret_cast<double*>(smem_tc + L.red);
  uint64_t* mma_bar = reinterpret_cast<uint64_t*>(smem_tc + L.bars);
  uint32_t* holder = reinterpret_cast<uint32_t*>(smem_tc + L.holder);
  __shared__ float s_bound[2];      // 2 eps max ||c_j||, e_c max ||c_j||^2
  __shared__ float2 s_pair[kTcThreads / 32];   // per-warp SSE pairs
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ntiles = (a.m + kTcRows - 1) / kTcRows;
  const int planeA = kb * kTcRows * 128, planeB = kb * N * 128;

  // ---- set-up: zero A (its K padding must stay finite), build B, cF, cc
  for (int q = tid; q < planes * planeA / 16; q += kTcThreads)
    reinterpret_cast<uint4*>(sA)[q] = make_uint4(0u, 0u, 0u, 0u);
  if constexpr (FP8) {
    // centroid j's scale 2^(7 - floor(log2 max|c_j|)) (1 for a zero or dead row)
    for (int j = tid; j < N; j += kTcThreads) {
      float mx = 0.f;
      if (j < k && a.mask[j])
        for (int f = 0; f < n; ++f) mx = fmaxf(mx, fabsf(__ldg(a.C + (size_t)j * a.cstride + f)));
      const int e2 = (mx > 0.f && mx <= 3.0e38f) ? max(ilogbf(mx), -119) : 7;
      csc[j] = ldexpf(1.f, e2 - 7);
    }
    __syncthreads();
    // K-major rows of 128 E4M3 features: byte f & 15 of 16-byte chunk
    // (f & 127) >> 4, 128-byte swizzled, K block f >> 7
    for (int e = tid; e < N * kb * 128; e += kTcThreads) {
      const int j = e / (kb * 128), f = e - j * (kb * 128);
      float v = 0.f;
      if (j < k && f < n && a.mask[j]) v = __ldg(a.C + (size_t)j * a.cstride + f);
      if (cf && j < k && f < n) cF[j * n + f] = v;
      const int w = f & 127, ch = w >> 4;
      const int off = (f >> 7) * N * 128 + (j >> 3) * 1024 + (j & 7) * 128 +
                      ((ch ^ (j & 7)) << 4) + (w & 15);
      sB[off] = (unsigned char)__nv_cvt_float_to_fp8(v / csc[j], __NV_SATFINITE, __NV_E4M3);
    }
  } else {
    for (int e = tid; e < N * kb * 64; e += kTcThreads) {
      const int j = e / (kb * 64), f = e - j * (kb * 64);
      float v = 0.f;
      if (j < k && f < n && a.mask[j]) v = __ldg(a.C + (size_t)j * a.cstride + f);
      if (cf && j < k && f < n) cF[j * n + f] = v;
      const int off = (f >> 6) * N * 128 + sw128_offset(j, f & 63);
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      *reinterpret_cast<__nv_bfloat16*>(sB + off) = h;
      if (planes == 2)
        *reinterpret_cast<__nv_bfloat16*>(sB + planeB + off) =
            __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
  float cmax = 0.f;
  for (int j = tid; j < N; j += kTcThreads) {
    float s = INFINITY;
    if (j < k && a.mask[j]) {
      s = 0.f;
      for (int f = 0; f < n; ++f) {
        const float c = __ldg(a.C + (size_t)j * a.cstride + f);
        s = fmaf(c, c, s);
      }
      cmax = fmaxf(cmax, s);
    }
    cc[j] = s;
  }
  // error of the tensor-core dot product relative to ||x|| ||c_j||: one BF16
  // rounding per operand, or (split form, hi*hi + hi*lo + lo*hi) the dropped
  // lo*lo term and the second roundings; plus FP32 accumulation
  const float eps = FP8 ? 1.01f * (0x1.0p-3f + 0x1.0p-8f + 0x1.0p-16f * sqrtf((float)n)) +
                               (float)(n + 16) * 0x1.0p-22f
                   : planes == 1 ? 1.01f * 0x1.0p-7f + (float)(n + 16) * 0x1.0p-22f
                                 : 3.1f * 0x1.0p-16f + (float)(3 * n + 16) * 0x1.0p-22f;
  cmax = warp_max_f32(cmax);
  if (lane == 0) red[warp] = cmax;
  for (int r = tid; r < kTcRows; r += kTcThreads) xx[r] = 0.f;
  if (tid == 0) {
    mbar_init(mma_bar, 1);
    for (int i = 0; i < S; ++i) mbar_init(sbar + i, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(holder, (uint32_t)a.ncols);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    float mx = 0.f;
    for (int w = 0; w < kTcThreads / 32; ++w) mx = fmaxf(mx, (float)red[w]);
    s_bound[0] = 2.f * eps * sqrtf(mx) * 1.0001f;
    s_bound[1] = (float)(n + 2) * 0x1.0p-22f * mx;
  }
  const uint32_t tmem = *holder;
  const uint32_t idesc = FP8 ? idesc_e4m3_f32(kTcRows, N) : idesc_bf16_f32(kTcRows, N);
  const float e_d = (float)(n + 4) * 0x1.0p-22f;    // exact FP32 distance vs true
  const bool xvec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
  const bool cvec = (n % 4 == 0) && (cf || ((a.cstride % 4 == 0) &&
                    ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0)));
  // the tile is converted in 16-byte chunks of 8 BF16: a row has kb * 8
  // chunk slots, of which the first nch = ceil(n / 8) hold data
  const int nch = (n + 7) >> 3;
  const int cshift = (nch <= 1) ? 0 : (nch <= 2) ? 1 : (nch <= 4) ? 2 : (nch <= 8) ? 3
                   : (nch <= 16) ? 4 : (nch <= 32) ? 5 : 6;   // log2 of chunk slots per row
  const int cslots = 1 << cshift;

  unsigned rescored = 0;
  bool ok = true;
  // bulk copy of this CTA's i-th tile into stage i % S (thread 0)
  auto issue = [&](long long i) {
    const long long tt = (long long)blockIdx.x + i * gridDim.x;
    if (tt >= ntiles) return;
    const int sidx = (int)(i % S);
    const int rr = (int)min((long long)kTcRows, a.m - tt * kTcRows);
    const uint32_t bytes = (uint32_t)(rr * n * 4);
    mbar_expect_tx(sbar + sidx, bytes);
    bulk_g2s(stg + (size_t)sidx * kTcRows * n, a.X + (size_t)tt * kTcRows * n, bytes, sbar + sidx);
  };
  if (tid == 0)
    for (long long i = 0; i < S; ++i) issue(i);
  for (long long it = 0;; ++it) {
    const long long t = (long long)blockIdx.x + it * gridDim.x;
    if (t >= ntiles) break;
    const long long r0 = t * kTcRows;
    const int rows = (int)min((long long)kTcRows, a.m - r0);
    const float* src = a.X + (size_t)r0 * n;
    const float* tile = S ? stg + (size_t)(it % S) * kTcRows * n : nullptr;
    if (S) {
      if (!mbar_wait(sbar + (it % S), (uint32_t)((it / S) & 1))) ok = false;
    } else if (tid == 0 && xvec) {   // pull my next tile into L2 while this one is processed
      const long long tn = t + gridDim.x;
      if ((tn + 1) * kTcRows <= a.m)
        prefetch_l2(a.X + (size_t)tn * kTcRows * n, (uint32_t)(kTcRows * n * 4));
    }

    if constexpr (FP8) {
      // ---- rows -> scaled E4M3, a warp per row: lane l holds the 8-feature
      // units l, l + 32, ... (n <= 512: at most two), so the row's maximum
      // and norm are warp reductions
      const int nunits = (n + 7) >> 3;
      for (int r = warp; r < kTcRows; r += kTcThreads / 32) {
        float v[2][8];
        float mx = 0.f, q = 0.f;
#pragma unroll
        for (int uu = 0; uu < 2; ++uu) {
          const int un = lane + 32 * uu, f0 = un * 8;
#pragma unroll
          for (int u = 0; u < 8; ++u) v[uu][u] = 0.f;
          if (r < rows && un < nunits) {
            const float* p = src + (size_t)r * n + f0;
            if (xvec && f0 + 8 <= n) {
              const float4 x0 = __ldg(reinterpret_cast<const float4*>(p));
              const float4 x1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
              v[uu][0] = x0.x; v[uu][1] = x0.y; v[uu][2] = x0.z; v[uu][3] = x0.w;
              v[uu][4] = x1.x; v[uu][5] = x1.y; v[uu][6] = x1.z; v[uu][7] = x1.w;
            } else {
#pragma unroll
              for (int u = 0; u < 8; ++u) if (f0 + u < n) v[uu][u] = __ldg(p + u);
            }
            if (xf) {   // FP32 copy for the exact distances
              float* d = xF + r * xs + f0;
              reinterpret_cast<float4*>(d)[0] = make_float4(v[uu][0], v[uu][1], v[uu][2], v[uu][3]);
              if (f0 + 8 <= xs)
                reinterpret_cast<float4*>(d)[1] = make_float4(v[uu][4], v[uu][5], v[uu][6], v[uu][7]);
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            mx = fmaxf(mx, fabsf(v[uu][u]));
            q = fmaf(v[uu][u], v[uu][u], q);
          }
        }
        mx = warp_max_f32(mx);
        q = warp_sum_f32(q);
        const int e2 = (mx > 0.f && mx <= 3.0e38f) ? max(ilogbf(mx), -119) : 7;
        const float inv = ldexpf(1.f, e2 - 7);   // 1 / scale, a power of two
        if (lane == 0) {
          xx[r] = q;
          rsc[r] = inv;
        }
#pragma unroll
        for (int uu = 0; uu < 2; ++uu) {
          const int un = lane + 32 * uu, f0 = un * 8;
          if (f0 >= kb * 128) continue;
          uint32_t w[2] = {0u, 0u};
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const uint32_t byte =
                (uint32_t)__nv_cvt_float_to_fp8(v[uu][u] / inv, __NV_SATFINITE, __NV_E4M3);
            w[u >> 2] |= byte << (8 * (u & 3));
          }
          const int wi = f0 & 127, ch = wi >> 4;
          const int off = (f0 >> 7) * (kTcRows * 128) + (r >> 3) * 1024 + (r & 7) * 128 +
                          ((ch ^ (r & 7)) << 4) + (wi & 8);
          *reinterpret_cast<uint2*>(sA + off) = make_uint2(w[0], w[1]);
        }
      }
    } else
    // ---- rows -> BF16 (hi[, lo]) 16-byte chunks; norms over the chunks of a row
    // (every thread runs cslots iterations; unrolled so that the loads of
    // several chunks are in flight together)
#pragma unroll 4
    for (int c = tid; c < kTcRows * cslots; c += kTcThreads) {
      const int r = c >> cshift, ch = c & (cslots - 1);
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = 0.f;
      const int f0 = ch * 8;
      if (S && r < rows && ch < nch) {   // from the staged tile (n % 4 == 0)
        const float4* p = reinterpret_cast<const float4*>(tile + (size_t)r * n + f0);
        const float4 x0 = p[0];
        v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
        if (f0 + 8 <= n) {
          const float4 x1 = p[1];
          v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
        }
      } else if (r < rows && ch < nch) {
        const float* p = src + (size_t)r * n + f0;
        if (xvec && f0 + 8 <= n) {
          const float4 x0 = __ldg(reinterpret_cast<const float4*>(p));
          const float4 x1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
          v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
          v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u) if (f0 + u < n) v[u] = __ldg(p + u);
        }
      }
      if (xf && r < rows && ch < nch) {   // FP32 copy for the exact distances
        float* d = xF + r * xs + f0;
        if (f0 + 8 <= xs) {
          reinterpret_cast<float4*>(d)[0] = make_float4(v[0], v[1], v[2], v[3]);
          reinterpret_cast<float4*>(d)[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {
          reinterpret_cast<float4*>(d)[0] = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
      float q = 0.f;
      uint32_t h[4], l[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        q = fmaf(v[2 * u], v[2 * u], q);
        q = fmaf(v[2 * u + 1], v[2 * u + 1], q);
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
        h[u] = *reinterpret_cast<const uint32_t*>(&hh);
        if (planes == 2) {
          const float2 hf = __bfloat1622float2(hh);
          const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * u] - hf.x, v[2 * u + 1] - hf.y);
          l[u] = *reinterpret_cast<const uint32_t*>(&ll);
        }
      }
      if (ch < kb * 8) {
        const int off = (ch >> 3) * (kTcRows * 128) + sw128_offset(r, (ch & 7) * 8);
        *reinterpret_cast<uint4*>(sA + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (planes == 2)
          *reinterpret_cast<uint4*>(sA + planeA + off) = make_uint4(l[0], l[1], l[2], l[3]);
      }
      // the cslots consecutive lanes of a row hold its partial norms; a row
      // wider than a warp leaves its second warp's sum in xx[kTcRows + r],
      // added to the first in that order by the epilogue
      const int span = cslots < 32 ? cslots : 32;
      for (int o = span >> 1; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if ((ch & 31) == 0) xx[(ch >> 5) * kTcRows + r] = q;
    }
    fence_proxy_async_smem();
    __syncthreads();
    BM_TC_TICK(0);
    // one stage: it is converted, so the next tile can start arriving now
    // (the epilogue then reads this tile's rows from global memory / L2)
    if (S == 1 && tid == 0) issue(it + 1);
    if (tid == 0) {
      tc_fence_after();
      const uint64_t da = sdesc_sw128(smem_u32(sA));
      const uint64_t db = sdesc_sw128(smem_u32(sB));
      const uint64_t alo = (uint64_t)(planeA >> 4), blo = (uint64_t)(planeB >> 4);
      uint32_t acc = 0;
      for (int b = 0; b < kb; ++b)
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t off = (uint64_t)((ks * 32) >> 4);
          const uint64_t ab = da + (uint64_t)((b * kTcRows * 128) >> 4) + off;
          const uint64_t bb = db + (uint64_t)((b * N * 128) >> 4) + off;
          if constexpr (FP8) {
            tc_mma_e4m3(tmem, ab, bb, idesc, acc);            // K = 32 per step
            acc = 1;
          } else {
            tc_mma_bf16(tmem, ab, bb, idesc, acc);            // hi * hi
            acc = 1;
            if (planes == 2) {
              tc_mma_bf16(tmem, ab, bb + blo, idesc, 1);      // hi * lo
              tc_mma_bf16(tmem, ab + alo, bb, idesc, 1);      // lo * hi
            }
          }
        }
      tc_commit(mma_bar);
    }
    if (!mbar_wait(mma_bar, (uint32_t)(it & 1))) ok = false;
    tc_fence_after();
    BM_TC_TICK(1);

    // ---- epilogue: one thread per row
    const int r = tid;
    const bool valid = r < rows;
    const float* xrow = S == 2 ? tile + (size_t)r * n : xf ? xF + r * xs : src + (size_t)r * n;
    // (the E4M3 conversion keeps a row's whole norm in xx[r]: a warp per row)
    const float xq =
        (!FP8 && cslots > 32 ? __fadd_rn(xx[r], xx[kTcRows + r]) : xx[r]) * 1.00002f;
    const float E1 = fmaf(sqrtf(xq), s_bound[0], s_bound[1]);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    // approximate distance minus ||x||^2 from accumulator column j (the E4M3
    // form scales the accumulator back by 1 / (row scale x centroid scale),
    // exact powers of two)
    const float s2 = FP8 ? -2.f * rsc[r] : -2.f;
    auto dapx = [&](float v, int j) {
      if constexpr (FP8) return fmaf(s2 * csc[j], v, cc[j]);
      else return fmaf(-2.f, v, cc[j]);
    };
    float m1 = INFINITY;
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tmem_ld32(lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (c0 + u < N) m1 = fminf(m1, dapx(v[u], c0 + u));
    }
    // every centroid that can hold the exact FP32 minimum lies within thr
    const float thr = m1 + 2.f * E1 + 3.f * e_d * fmaxf(0.f, xq + m1 + E1);
    BM_TC_TICK(2);
    float best = INFINITY;
    int bj = INT_MAX, ncand = 0;
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tmem_ld32(lane_base + (uint32_t)c0, v);
      uint32_t cand = 0u;
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (c0 + u < k && dapx(v[u], c0 + u) <= thr) cand |= 1u << u;
      if (!valid) cand = 0u;
      // exact distances of the candidates, ascending index
      while (cand) {
        const int j = c0 + __ffs(cand) - 1;
        cand &= cand - 1u;
        ++ncand;
        const float* crow = cf ? cF + j * n : a.C + (size_t)j * a.cstride;
        const float d = dist_exact(xrow, crow, n, (xf || xvec) && cvec);
        if (bj == INT_MAX || d < best) { best = d; bj = j; }
      }
    }
    // the tile's SSE as an exact (hi, lo) pair, so that the total does not
    // depend on how tiles are spread over CTAs
    float th = valid ? best : 0.f, tl = 0.f;
    if (valid) {
      if (BM_GUARD(r0 + r < a.m, a.status)) {
        if (a.labels) a.labels[r0 + r] = bj;
        if (a.dmin) a.dmin[r0 + r] = best;
      }
      rescored += ncand > 1;
    }
    warp_two_sum(th, tl);
    if (lane == 0) s_pair[warp] = make_float2(th, tl);
    xx[r] = 0.f;
    BM_TC_TICK(3);
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      float2 p = s_pair[0];
      for (int w = 1; w < kTcThreads / 32; ++w) {
        two_sum_acc(p.x, p.y, s_pair[w].x);
        p.y = __fadd_rn(p.y, s_pair[w].y);
      }
      a.part[t] = p;
      // two stages: this tile's stage has been read for the last time
      if (S == 2) {
        fence_proxy_async_smem();
        issue(it + 2);
      }
    }
    BM_TC_TICK(4);
  }

  // ---- SSE: the last CTA adds the per-tile pairs in tile order (TwoSum)
  const unsigned resc = __reduce_add_sync(0xffffffffu, rescored);
  if (lane == 0 && resc) atomicAdd(a.rescored, (unsigned long long)resc);
  if (!ok) atomicCAS(a.status, 0, kStatusTimeout);
  __syncthreads();
  __shared__ int s_last;
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    float hi = 0.f, lo = 0.f;
    for (long long q = tid; q < ntiles; q += kTcThreads) {
      const float2 p = __ldcg(a.part + q);
      two_sum_acc(hi, lo, p.x);
      lo = __fadd_rn(lo, p.y);
    }
    warp_two_sum(hi, lo);
    if (lane == 0) s_pair[warp] = make_float2(hi, lo);
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < kTcThreads / 32; ++w) tot += (double)s_pair[w].x + (double)s_pair[w].y;
      *a.sse = tot;
      *a.ticket = 0u;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)a.ncols);
}

size_t assign_tc_smem(int n, int k, int terms, int* stages_out, int* kb_out,
                      int* npad16_out, int* ncols_out, int* cf_out, bool bulk_ok,
                      size_t limit) {
  const bool fp8 = terms == kTermsFp8;
  const int kb = fp8 ? (n + 127) / 128 : (n + 63) / 64;   // K blocks of 128-byte rows
  const int npad16 = (k + 15) / 16 * 16;
  const int planes = terms == 3 ? 2 : 1;
  int ncols = 32;
  while (ncols < npad16) ncols <<= 1;
  const bool cf = k * n * 4 <= 24 * 1024;
  // two staged tiles when they fit, else thread loads: with a single stage
  // the CTA has to read the rows back from L2 for the exact distances, and
  // the larger footprint leaves fewer CTAs per SM to hide that latency
  // (measured slower than thread loads at n = 128)
  int stages = 0;
  if (!fp8 && bulk_ok && n % 4 == 0 &&
      (size_t)tc_layout(n, kb, npad16, k, planes, cf, 2).total + 1024 <= limit)
    stages = 2;   // (the E4M3 form converts from its own thread loads)
  const TcLayout L = tc_layout(n, kb, npad16, k, planes, cf, stages);
  *stages_out = stages;
  *kb_out = kb;
  *npad16_out = npad16;
  *ncols_out = ncols;
  *cf_out = cf;
  return (size_t)L.total + 1024;   // + alignment slack of the dynamic base
}

template <bool FP8>
static int assign_tc_max_grid_t(size_t smem) {
  auto fn = assign_tc_kernel<FP8>;
  if (allow_max_smem(fn) != cudaSuccess) return 0;
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
  int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  const size_t per_cta = smem + fa.sharedSizeBytes + 1024;   // + reserved per CTA
  int by_smem = (int)((size_t)smem_sm / per_cta);
  int by_regs = regs_sm / std::max(1, fa.numRegs * kTcThreads);
  int per_sm = std::min(std::min(by_smem, by_regs), 8);
  if (per_sm < 1) return 0;
  return per_sm * sms;
}

// CTAs per SM from shared memory and registers (the occupancy API reports a
// single CTA per SM for this TMEM-allocating kernel, but more co-reside; the
// host additionally caps the count by TMEM columns).
int assign_tc_max_grid(size_t smem, int terms) {
  return terms == kTermsFp8 ? assign_tc_max_grid_t<true>(smem)
                            : assign_tc_max_grid_t<false>(smem);
}

cudaError_t launch_assign_tc(const AssignTcArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (a.terms == kTermsFp8) {
    cudaError_t e = allow_max_smem(assign_tc_kernel<true>);
    if (e != cudaSuccess) return e;
    assign_tc_kernel<true><<<grid, kTcThreads, smem, st>>>(a);
  } else {
    cudaError_t e = allow_max_smem(assign_tc_kernel<false>);
    if (e != cudaSuccess) return e;
    assign_tc_kernel<false><<<grid, kTcThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace bm
