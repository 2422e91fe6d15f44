// Tensor-core chunk kernel: Alg. 1's loop body (gather, K-means++ reseed of
// Sec. 3.3 with three candidates per Sec. 5, Lloyd iterations of Sec. 2 with
// the stop rule of Sec. 5, keep-the-best) for rows wider than 32 features,
// with the Eq. 1 distances of every Lloyd assignment on the 5th-generation
// tensor cores and exact FP32 rescoring.
//
// One cooperative launch per chunk, one CTA per SM, 256 threads; CTA b owns
// sample rows [b R, b R + R).  Per Lloyd iteration a CTA
//   A.  streams its rows in 128-row tiles and 64-feature blocks: the FP32 rows
//       become split-BF16 (hi, lo) planes in a 128-byte-swizzled K-major
//       tile, the centroid planes of the block arrive by a bulk copy from a
//       pre-swizzled global copy (written where the centroids change), and
//       tcgen05.mma accumulates hi*hi + hi*lo + lo*hi into TMEM.  The
//       epilogue (8 warps: TMEM lane quarter x column half) bounds every
//       approximate distance (see the tensor-core assignment) and records
//       the candidate centroids of each row;
//   A'. decides the rows with more than one candidate from exact FP32
//       distances (a half-warp per row, coalesced loads);
//   BC. sweeps its rows again in feature blocks staged in shared memory:
//       the exact FP32 distance of every single-candidate
//       row to its centroid (four partial sums over f mod 4, ascending f --
//       the arithmetic of the FP32 kernels), and, over the rows sorted by
//       label (stable counting sort), the per-centroid sums of (p - c) that
//       the update needs, written as this CTA's partials.
// A grid barrier, the reduction of the partials (one warp per centroid and
// 32-feature slice, which also writes the new BF16 planes and the squared
// norms of the slice), a second grid barrier.  Every sum has a fixed order,
// so results are reproducible for a given grid.
//
// K-means++ uses the same pieces: D^2 is the assignment's distance, and the
// candidates' distances come from the staged sweep.
//
// Screening arithmetic (tc_planes, tc_fp8): BF16 products (one plane), split
// BF16 (two planes), or E4M3 products with FP32 accumulation in K blocks of
// 128 features.  In the E4M3 form each own row is scaled by the power of two
// that brings its largest magnitude into [128, 256), and every centroid of
// the chunk by one power of two cs chosen the same way from M, the largest
// magnitude over the sample rows and the live incumbent centroids (every
// centroid the chunk produces is a sample row or a mean of sample rows, so
// |c_f| <= M up to rounding and nothing saturates).  The scales are exact,
// so the epilogue scales the accumulator back with one factor per row.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "bm_chunk_common.cuh"
#include "bm_device.cuh"
#include "bm_internal.h"
#include "bm_kpp.cuh"
#include "bm_tc.cuh"

namespace bm {

constexpr int kTccThreads = 256;
constexpr int kTccM = 128;           // MMA M: rows per tile
constexpr int kTccWarps = kTccThreads / 32;

struct TccLayout {
  int ring_a, ring_b, ring_slot, stage_c, sstride;
  int region, cmask, lab, dmin, part4, dc, order, cnt, start, cur, wc, cand, live, lidx, cc,
      xx, rsc, xm, mlist, red, bars, holder, total;
};

// Shared-memory layout.  The region at offset 0 holds either the ns-slot
// MMA ring (A block: 128 rows x 128 bytes x `planes` planes; B block: n16
// rows x 128 bytes x `planes` planes) or the staged feature block of the
// exact passes (R rows and k centroid rows of fb floats, row stride fb + 4).
__host__ __device__ inline TccLayout tcc_layout(int npad, int k, int R, int n16, int fb,
                                                int ns, int planes) {
  TccLayout L;
  L.ring_a = planes * kTccM * 128;
  L.ring_b = planes * n16 * 128;
  L.ring_slot = L.ring_a + L.ring_b;
  L.sstride = fb + 4;
  L.stage_c = align_up(R * L.sstride * 4, 16);
  const int stage = L.stage_c + k * L.sstride * 4;
  int o = align_up(ns * L.ring_slot > stage ? ns * L.ring_slot : stage, 1024);
  L.region = 0;
  L.cmask = o;  o += R * 16;                             // candidate bits, 4 words per row
  L.lab = o;    o += align_up(R * 4, 16);
  L.dmin = o;   o += align_up(R * 4, 16);
  L.part4 = o;  o += kMaxTrials * R * 16;                // partial distance sums
  L.dc = o;     o += align_up(kMaxTrials * R * 4, 16);
  L.order = o;  o += align_up(R * 4, 16);                // rows sorted by label
  L.cnt = o;    o += align_up(k * 4, 16);
  L.start = o;  o += align_up((k + 1) * 4, 16);
  L.cur = o;    o += align_up(k * 4, 16);
  L.wc = o;     o += align_up(kTccWarps * k * 4, 16);
  L.cand = o;   o += align_up(kMaxTrials * npad * 4, 16);
  L.live = o;   o += align_up(k * 4, 16);
  L.lidx = o;   o += align_up((k + 1) * 4, 16);
  L.cc = o;     o += align_up(n16 * 4, 16);
  L.xx = o;     o += align_up(R * 4, 16);                // ||x||^2 of own rows
  L.rsc = o;    o += align_up(R * 4, 16);                // E4M3: 1 / scale of own rows
  L.xm = o;     o += 2 * kTccM * 4;                      // column-half minima
  L.mlist = o;  o += align_up((R + 1) * 4, 16);          // multi-candidate rows
  L.red = o;    o += 80 * 8;
  L.bars = o;   o += 8 * 8;
  L.holder = o; o += 16;
  L.total = o;
  return L;
}

// Shared-memory view of one CTA.
struct TccS {
  unsigned char* ring;
  float* sP;          // staged rows [R][sstride]
  float* sC;          // staged centroids [k][sstride]
  uint32_t* cmask;    // [R][4]
  int* lab;
  float* dmin;
  float* part4;       // [kMaxTrials][R][4]
  float* dc;          // [kMaxTrials][R]
  int* order;
  int* cnt;
  int* start;
  int* cur;
  int* wc;            // [warps][k]
  float* cand;        // [kMaxTrials][npad]
  int* live;
  int* lidx;
  float* cc;          // [n16] ||c_j||^2, +inf if not live
  float* xx;          // [R] ||x||^2 of own rows
  float* rsc;         // [R] E4M3 form: 1 / scale of own rows (a power of two)
  float* xm;          // [2][128]
  int* mlist;         // [R + 1], count at [R]
  double* red;
  uint64_t* bfull;    // [ns] the A and B blocks of a ring slot arrived
  uint64_t* sfree;    // [ns] the MMAs reading a ring slot finished
  uint64_t* accb;     // accumulator complete
  uint32_t* holder;
  int sstride;
  int ring_slot, ring_a, ns;
};

// Pipeline counters (uniform across the CTA): ring steps, tiles.
struct TccPipe {
  uint32_t ring, acc;
};

struct TccBound {
  float b0, b1;       // 2 eps max ||c|| (+ the E4M3 underflow term), (n + 2) 2^-22 max ||c||^2
};

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---------------------------------------------------------------- centroids
// E4M3 form: the chunk's centroid scale cs, 1 / cs and M (the largest
// magnitude it was chosen from), the same in every CTA.
__device__ __forceinline__ float* fp8_cscale() {
  __shared__ float v[3];
  return v;
}

// Writes centroid value v of (j, f) into the global centroid operand: the
// BF16 planes (hi, lo), or the E4M3 byte of v cs.
__device__ __forceinline__ void put_cb(const ChunkArgs& a, int j, int f, float v) {
  const int n16 = a.tc_n16;
  if (a.tc_fp8) {
    const int w = f & 127;
    const int off = (f >> 7) * (n16 * 128) + (j >> 3) * 1024 + (j & 7) * 128 +
                    (((w >> 4) ^ (j & 7)) << 4) + (w & 15);
    a.Cb[off] = (unsigned char)__nv_cvt_float_to_fp8(v * fp8_cscale()[0], __NV_SATFINITE,
                                                     __NV_E4M3);
    return;
  }
  const int off = (f >> 6) * (2 * n16 * 128) + sw128_offset(j, f & 63);
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16*>(a.Cb + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(a.Cb + off + n16 * 128) =
      __float2bfloat16_rn(v - __bfloat162float(h));
}

// Centroid j, features [32 q, 32 q + 32) held one per lane (value v of lane
// l is feature 32 q + l) -> C (when write_c), the planes and the squared
// norms of the four 8-feature slices (sum over the slice's lanes in a fixed
// order).
__device__ __forceinline__ void publish32(const ChunkArgs& a, int j, int q, float v,
                                          bool write_c) {
  const int l = threadIdx.x & 31, f = q * 32 + l;
  const int nsl = (a.npad + 7) >> 3;
  const bool on = f < a.n;
  if (on) {
    if (write_c) a.C[(size_t)j * a.npad + f] = v;
    put_cb(a, j, f, v);
  }
  float sq = on ? v * v : 0.f;
  sq += __shfl_xor_sync(0xffffffffu, sq, 1);
  sq += __shfl_xor_sync(0xffffffffu, sq, 2);
  sq += __shfl_xor_sync(0xffffffffu, sq, 4);
  const int sl = q * 4 + (l >> 3);
  if ((l & 7) == 0 && sl < nsl) a.sqs[(size_t)j * nsl + sl] = sq;
}

// cc[j] and the error-bound constants from the slice norms (after a grid
// barrier); dead and padding columns get +inf.
__device__ void load_norms(const ChunkArgs& a, const TccS& S, TccBound* bd) {
  const int nsl = (a.npad + 7) >> 3;
  float cmax = 0.f;
  for (int j = threadIdx.x; j < a.tc_n16; j += blockDim.x) {
    float s = INFINITY;
    if (j < a.k && S.live[j]) {
      s = 0.f;
      for (int c = 0; c < nsl; ++c) s += __ldcg(a.sqs + (size_t)j * nsl + c);
      cmax = fmaxf(cmax, s * 1.0001f);
    }
    S.cc[j] = s;
  }
  cmax = warp_max_f32(cmax);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) S.red[w] = cmax;
  __syncthreads();
  float mx = 0.f;
  for (int i = 0; i < kTccWarps; ++i) mx = fmaxf(mx, (float)S.red[i]);
  // one BF16 rounding per operand, or for split BF16 products the dropped
  // lo*lo term and the second roundings; plus FP32 accumulation over n
  // products.  E4M3: each scaled operand is within 2^-4 relative or 2^-10
  // absolute (the subnormal spacing) of its value, so with row scale
  // 2^(7 - e) (2^e <= max|x_f| <= ||x||) and centroid scale cs (M cs < 256)
  //   |x~ c~ - x c| <= ||x|| ||c|| (2^-3 + 2^-8 + 1.07 2^-17 sqrt n)
  //                  + ||x|| M (1.07 2^-17 sqrt n + n 2^-34),
  // plus the accumulation over n products of at most 1.14 ||x|| ||c||.
  const float rn = sqrtf((float)a.n);
  const float eps =
      a.tc_fp8 ? 0x1.0p-3f + 0x1.0p-8f + 1.07f * 0x1.0p-17f * rn +
                     1.14f * (float)(a.n + 16) * 0x1.0p-22f
      : a.tc_planes == 1 ? 1.01f * 0x1.0p-7f + (float)(a.n + 16) * 0x1.0p-22f
                         : 3.1f * 0x1.0p-16f + (float)(3 * a.n + 16) * 0x1.0p-22f;
  const float tau = a.tc_fp8 ? 1.01f * (1.07f * 0x1.0p-17f * rn + (float)a.n * 0x1.0p-34f) : 0.f;
  bd->b0 = 2.f * (eps * sqrtf(mx) + (a.tc_fp8 ? tau * fp8_cscale()[2] : 0.f)) * 1.0001f;
  bd->b1 = (float)(a.n + 2) * 0x1.0p-22f * mx;
  __syncthreads();
}

// ---------------------------------------------------------------- planes
// Own rows -> BF16 tiles in global memory, once per chunk (P does not
// change across Lloyd iterations): tile t, K block kb of this CTA is one
// contiguous block of 16 KB per plane (the hi plane, then for split BF16 the
// lo plane) in the 128-byte-swizzled K-major layout of the MMA; ||x||^2 of
// every own row -> S.xx.
// E4M3 form: own rows -> E4M3 tiles (K blocks of 128 features).  A first
// pass gives each row its largest magnitude and norm (8 threads per row,
// every float4 of the row in flight at once); row i is scaled by
// 1 / rsc[i], the power of two that brings that magnitude into [128, 256).
// A second pass converts 16-feature chunks (4 per thread in flight) into
// the 128-byte-swizzled K-major tiles; padding rows and features are zero.
// Returns the largest magnitude over own rows (every thread).
__device__ float tcc_convert_own_fp8(const ChunkArgs& a, const TccS& S, int r0, int nrows) {
  const int tid = threadIdx.x, kb = a.tc_kb, npad = a.npad, np4 = npad >> 2;
  constexpr int blk = kTccM * 128;
  const float4* P4 = reinterpret_cast<const float4*>(a.P) + (size_t)r0 * np4;
  float cmax = 0.f;
  for (int i0 = 0; i0 < nrows; i0 += kTccThreads / 8) {
    const int i = i0 + (tid >> 3), c = tid & 7;
    float4 v[16];   // np4 <= 128
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int q = c + 8 * u;
      v[u] = (i < nrows && q < np4) ? __ldcg(P4 + (size_t)i * np4 + q)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float mx = 0.f, nq = 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
      nq = fmaf(v[u].x, v[u].x, nq);
      nq = fmaf(v[u].y, v[u].y, nq);
      nq = fmaf(v[u].z, v[u].z, nq);
      nq = fmaf(v[u].w, v[u].w, nq);
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {   // the 8 threads of a row are consecutive lanes
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      nq += __shfl_xor_sync(0xffffffffu, nq, o);
    }
    if (c == 0 && i < nrows) {
      const int e2 = (mx > 0.f && mx <= 3.0e38f) ? max(ilogbf(mx), -119) : 7;
      S.xx[i] = nq;
      S.rsc[i] = ldexpf(1.f, e2 - 7);
    }
    cmax = fmaxf(cmax, mx);
  }
  __syncthreads();
  unsigned char* base = a.Pb + (size_t)blockIdx.x * a.tc_tpc * kb * blk;
  for (int t0 = 0; t0 < nrows; t0 += kTccM) {
    const int rows = min(kTccM, nrows - t0);
    for (int b = 0; b < kb; ++b) {
      unsigned char* dst = base + (size_t)((t0 / kTccM) * kb + b) * blk;
      float4 v[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = tid + u * kTccThreads, r = q >> 3, f0 = b * 128 + (q & 7) * 16;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          v[u][e] = (r < rows && f0 + 4 * e < npad)
              ? __ldcg(P4 + (size_t)(t0 + r) * np4 + (f0 >> 2) + e)
              : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = tid + u * kTccThreads, r = q >> 3, ch = q & 7;
        const float inv = r < rows ? S.rsc[t0 + r] : 1.f;
        uint32_t wd[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4 x = v[u][e];
          wd[e] = (uint32_t)__nv_cvt_float_to_fp8(x.x / inv, __NV_SATFINITE, __NV_E4M3) |
                  ((uint32_t)__nv_cvt_float_to_fp8(x.y / inv, __NV_SATFINITE, __NV_E4M3) << 8) |
                  ((uint32_t)__nv_cvt_float_to_fp8(x.z / inv, __NV_SATFINITE, __NV_E4M3) << 16) |
                  ((uint32_t)__nv_cvt_float_to_fp8(x.w / inv, __NV_SATFINITE, __NV_E4M3) << 24);
        }
        const int off = (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
        *reinterpret_cast<uint4*>(dst + off) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      }
    }
  }
  fence_proxy_async_global();   // the tiles are read back by bulk copies
  const int w = tid >> 5, l = tid & 31;
  const float m = warp_max_f32(cmax);
  __syncthreads();
  if (l == 0) S.red[w] = m;
  __syncthreads();
  float all = 0.f;
  for (int i = 0; i < kTccWarps; ++i) all = fmaxf(all, (float)S.red[i]);
  __syncthreads();
  return all;
}

__device__ void tcc_convert_own(const ChunkArgs& a, const TccS& S, int r0, int nrows) {
  const int tid = threadIdx.x, kb = a.tc_kb, npad = a.npad;
  const int blk = a.tc_planes * kTccM * 128;
  for (int i = tid; i < nrows; i += blockDim.x) S.xx[i] = 0.f;
  __syncthreads();
  unsigned char* base = a.Pb + (size_t)blockIdx.x * a.tc_tpc * kb * blk;
  for (int t0 = 0; t0 < nrows; t0 += kTccM) {
    const int rows = min(kTccM, nrows - t0);
    const float* src = a.P + (size_t)(r0 + t0) * npad;
    for (int b = 0; b < kb; ++b) {
      unsigned char* dst = base + (size_t)((t0 / kTccM) * kb + b) * blk;
      // 8 threads per row, one 8-feature chunk each
      float v[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = tid + u * kTccThreads;
        const int r = c >> 3, f0 = b * 64 + (c & 7) * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[u][e] = 0.f;
        if (r < rows && f0 < npad) {
          const float4* p = reinterpret_cast<const float4*>(src + (size_t)r * npad + f0);
          const float4 x0 = __ldcg(p);
          v[u][0] = x0.x; v[u][1] = x0.y; v[u][2] = x0.z; v[u][3] = x0.w;
          if (f0 + 4 < npad) {
            const float4 x1 = __ldcg(p + 1);
            v[u][4] = x1.x; v[u][5] = x1.y; v[u][6] = x1.z; v[u][7] = x1.w;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = tid + u * kTccThreads;
        const int r = c >> 3, ch = c & 7;
        float nq = 0.f;
        uint32_t h[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          nq = fmaf(v[u][2 * e], v[u][2 * e], nq);
          nq = fmaf(v[u][2 * e + 1], v[u][2 * e + 1], nq);
          const __nv_bfloat162 hh = __floats2bfloat162_rn(v[u][2 * e], v[u][2 * e + 1]);
          const float2 hf = __bfloat1622float2(hh);
          const __nv_bfloat162 ll = __floats2bfloat162_rn(v[u][2 * e] - hf.x,
                                                          v[u][2 * e + 1] - hf.y);
          h[e] = *reinterpret_cast<const uint32_t*>(&hh);
          lo[e] = *reinterpret_cast<const uint32_t*>(&ll);
        }
        const int off = sw128_offset(r, ch * 8);
        *reinterpret_cast<uint4*>(dst + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (a.tc_planes == 2)
          *reinterpret_cast<uint4*>(dst + kTccM * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        // the 8 threads of a row are consecutive lanes
        nq += __shfl_xor_sync(0xffffffffu, nq, 1);
        nq += __shfl_xor_sync(0xffffffffu, nq, 2);
        nq += __shfl_xor_sync(0xffffffffu, nq, 4);
        if (ch == 0 && r < rows) S.xx[t0 + r] += nq;
      }
    }
  }
  fence_proxy_async_global();   // the tiles are read back by bulk copies
  __syncthreads();
}

// ---------------------------------------------------------------- pass A
// Candidates of own rows against the live centroids: for each row, the bits
// of the centroids whose bounded approximate distance can hold the exact
// minimum; single-candidate rows get their label.  The (tile, K block)
// steps move through an ns-slot ring: warp 1 issues the bulk copies (row
// planes of the step, centroid planes of its K block) as slots free up,
// running up to ns steps ahead -- into the next tile while this tile's MMAs
// and epilogue run -- and thread 0 issues the MMAs as blocks arrive.
__device__ bool tcc_pass_a(const ChunkArgs& a, const TccS& S, int r0, int nrows,
                           const TccBound& bd, uint32_t tmem, TccPipe& pp) {
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int kb = a.tc_kb, N = a.tc_n16, ns = S.ns;
  const bool fp8 = a.tc_fp8 != 0;
  const uint32_t idesc = fp8 ? idesc_e4m3_f32(kTccM, N) : idesc_bf16_f32(kTccM, N);
  const float e_d = (float)(a.n + 4) * 0x1.0p-22f;
  const int planes = a.tc_planes;
  const uint32_t abytes = planes * kTccM * 128, bbytes = planes * N * 128;
  // the global BF16 centroid planes keep both (hi, lo); E4M3 has one
  const size_t cb_stride = (fp8 ? 1 : 2) * (size_t)N * 128;
  const unsigned char* pbase = a.Pb + (size_t)blockIdx.x * a.tc_tpc * kb * abytes;
  const int ntl = (nrows + kTccM - 1) / kTccM;
  const uint32_t first = pp.ring, total = (uint32_t)(ntl * kb);
  uint32_t issued = first;   // producer warp's count of issued steps
  bool ok = true;
  if (w == 1 && lane == 0) fence_proxy_async_global();
  for (int t = 0; t < ntl; ++t) {
    const int t0 = t * kTccM, rows = min(kTccM, nrows - t0);
    if (w == 1) {
      // producer: the rest of this tile and the first steps of the next;
      // a slot is reused once the MMAs of its previous step have completed
      const uint32_t limit = min(first + (uint32_t)((t + 1) * kb + ns), first + total);
      for (; issued < limit; ++issued) {
        const uint32_t q = issued, sl = q % (uint32_t)ns, use = q / (uint32_t)ns;
        if (use > 0 && !mbar_wait(S.sfree + sl, (use - 1u) & 1u)) ok = false;
        if (lane == 0) {
          const int st = (int)(q - first), tt = st / kb, b = st - tt * kb;
          unsigned char* sa = S.ring + sl * S.ring_slot;
          mbar_expect_tx(S.bfull + sl, abytes + bbytes);
          bulk_g2s(sa, pbase + (size_t)(tt * kb + b) * abytes, abytes, S.bfull + sl);
          bulk_g2s(sa + S.ring_a, a.Cb + (size_t)b * cb_stride, bbytes, S.bfull + sl);
        }
        __syncwarp();
      }
    }
    if (tid == 0) {
      for (int b = 0; b < kb; ++b) {
        const uint32_t q = first + (uint32_t)(t * kb + b);
        const uint32_t sl = q % (uint32_t)ns, use = q / (uint32_t)ns;
        if (!mbar_wait(S.bfull + sl, use & 1u)) ok = false;
        tc_fence_after();
        unsigned char* sa = S.ring + sl * S.ring_slot;
        const uint64_t da = sdesc_sw128(smem_u32(sa));
        const uint64_t db = sdesc_sw128(smem_u32(sa + S.ring_a));
        const uint64_t alo = (uint64_t)((kTccM * 128) >> 4), blo = (uint64_t)((N * 128) >> 4);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {   // 32 bytes of K per step: 16 BF16 or 32 E4M3
          const uint64_t off = (uint64_t)((ks * 32) >> 4);
          if (fp8) {
            tc_mma_e4m3(tmem, da + off, db + off, idesc, (b > 0 || ks > 0) ? 1u : 0u);
            continue;
          }
          tc_mma_bf16(tmem, da + off, db + off, idesc, (b > 0 || ks > 0) ? 1u : 0u);
          if (planes == 2) {
            tc_mma_bf16(tmem, da + off, db + blo + off, idesc, 1u);
            tc_mma_bf16(tmem, da + alo + off, db + off, idesc, 1u);
          }
        }
        tc_commit(S.sfree + sl);
        if (b == kb - 1) tc_commit(S.accb);
      }
    }
    __syncwarp();
    if (!mbar_wait(S.accb, pp.acc & 1u)) ok = false;
    ++pp.acc;
    tc_fence_after();
    __syncwarp();

    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .., column half w / 4
    const int qd = w & 3, hf = w >> 2;
    const int r = qd * 32 + lane;
    const bool valid = r < rows;
    const uint32_t lane_base = tmem + ((uint32_t)(qd * 32) << 16);
    // -2 x.c from the accumulator: E4M3 scales it back by 1 / (row scale x
    // cs), exact powers of two
    const float g = fp8 && valid ? -2.f * S.rsc[t0 + r] * fp8_cscale()[1] : -2.f;
    float m1 = INFINITY;
    for (int c0 = hf * 32; c0 < N; c0 += 64) {
      float acc[32];
      tmem_ld32(lane_base + (uint32_t)c0, acc);
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (c0 + u < N) m1 = fminf(m1, fmaf(g, acc[u], S.cc[c0 + u]));
    }
    S.xm[hf * kTccM + r] = m1;
    __syncthreads();
    m1 = fminf(S.xm[r], S.xm[kTccM + r]);
    const float xq = (valid ? S.xx[t0 + r] : 0.f) * 1.00002f;
    const float E1 = fmaf(sqrtf(xq), bd.b0, bd.b1);
    const float thr = m1 + 2.f * E1 + 3.f * e_d * fmaxf(0.f, xq + m1 + E1);
    const int i = t0 + r;
    for (int c0 = hf * 32; c0 < N; c0 += 64) {
      float acc[32];
      tmem_ld32(lane_base + (uint32_t)c0, acc);
      uint32_t bits = 0u;
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (c0 + u < N && S.cc[c0 + u] < INFINITY && fmaf(g, acc[u], S.cc[c0 + u]) <= thr)
          bits |= 1u << u;
      if (valid) S.cmask[i * 4 + (c0 >> 5)] = bits;
    }
    if (valid && hf == 0)   // words beyond N stay empty
      for (int c0 = ((N + 31) >> 5) * 32; c0 < 128; c0 += 32) S.cmask[i * 4 + (c0 >> 5)] = 0u;
    tc_fence_before();
    __syncthreads();
    if (valid && hf == 0) {
      int nc = 0, j = INT_MAX;
#pragma unroll
      for (int wd = 0; wd < 4; ++wd) {
        const uint32_t m = S.cmask[i * 4 + wd];
        nc += __popc(m);
        if (m && j == INT_MAX) j = wd * 32 + __ffs(m) - 1;
      }
      S.lab[i] = nc == 1 ? j : (nc == 0 ? INT_MAX : -1);   // -1: decided in pass A'
      if (nc == 0) S.dmin[i] = INFINITY;   // no live centroid (or non-finite data)
    }
    __syncthreads();
  }
  pp.ring = first + total;
  return ok;
}

// ---------------------------------------------------------------- pass A'
// Rows with several candidates: exact FP32 distances to each candidate, a
// half-warp per row, lowest index on ties.
__device__ void tcc_pass_multi(const ChunkArgs& a, const TccS& S, int r0, int nrows) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, npad = a.npad;
  if (threadIdx.x == 0) S.mlist[a.rows_per_cta] = 0;
  __syncthreads();
  for (int i0 = 0; i0 < nrows; i0 += kTccThreads) {
    const int i = i0 + threadIdx.x;
    const bool multi = i < nrows && S.lab[i] == -1;
    const unsigned bal = __ballot_sync(0xffffffffu, multi);
    int base = 0;
    if (l == 0 && bal) base = atomicAdd(S.mlist + a.rows_per_cta, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (multi) S.mlist[base + __popc(bal & ((1u << l) - 1u))] = i;
  }
  __syncthreads();
  const int nm = S.mlist[a.rows_per_cta];
  // a half-warp per row, so two rows (and their candidates' centroid rows)
  // are in flight per warp: lane h of half hw holds features 4 h + 64 u
  // (u < 8: npad <= 512)
  const int h = l & 15, hw = l >> 4, nu = (npad + 63) >> 6;
  for (int e0 = 2 * w; e0 < nm; e0 += 2 * kTccWarps) {
    const int e = e0 + hw;
    const bool on = e < nm;
    const int i = on ? S.mlist[e] : 0;
    float4 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int f = 4 * h + 64 * u;
      x[u] = (on && u < nu && f < npad)
          ? __ldcg(reinterpret_cast<const float4*>(a.P + (size_t)(r0 + i) * npad + f))
          : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    uint32_t mw[4];
#pragma unroll
    for (int wd = 0; wd < 4; ++wd) mw[wd] = on ? S.cmask[i * 4 + wd] : 0u;
    float best = INFINITY;
    int bj = INT_MAX, wd = 0;
    while (true) {
      // the next (up to) two candidates of this half's row, ascending; the
      // warp runs while either half has some left (the sums shuffle across it)
      int js[2] = {0, 0}, nj = 0;
      while (nj < 2 && wd < 4) {
        if (mw[wd] == 0u) { ++wd; continue; }
        js[nj++] = wd * 32 + __ffs(mw[wd]) - 1;
        mw[wd] &= mw[wd] - 1u;
      }
      if ((nj | __shfl_xor_sync(0xffffffffu, nj, 16)) == 0) break;
      float4 cv[2][8];
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int f = 4 * h + 64 * u;
          cv[t][u] = (t < nj && u < nu && f < npad)
              ? __ldcg(reinterpret_cast<const float4*>(a.C + (size_t)js[t] * npad + f))
              : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (u >= nu) break;
          const float e0 = x[u].x - cv[t][u].x, e1 = x[u].y - cv[t][u].y;
          const float e2 = x[u].z - cv[t][u].z, e3 = x[u].w - cv[t][u].w;
          s0 = fmaf(e0, e0, s0);
          s1 = fmaf(e1, e1, s1);
          s2 = fmaf(e2, e2, s2);
          s3 = fmaf(e3, e3, s3);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {   // within the half-warp
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          s2 += __shfl_xor_sync(0xffffffffu, s2, o);
          s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        }
        const float d = (s0 + s1) + (s2 + s3);
        if (t < nj && (bj == INT_MAX || d < best)) { best = d; bj = js[t]; }
      }
    }
    if (on && h == 0) {
      S.lab[i] = bj;
      S.dmin[i] = best;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- sort
// Stable counting sort of own rows by label: order[start[j] ..) lists the
// rows of centroid j in ascending row order; cnt[j] members.
__device__ void tcc_sort(const ChunkArgs& a, const TccS& S, int nrows) {
  const int k = a.k, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int j = threadIdx.x; j < k; j += blockDim.x) S.cnt[j] = 0;
  for (int q = threadIdx.x; q < kTccWarps * k; q += blockDim.x) S.wc[q] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    const int j = S.lab[i];
    if (j >= 0 && j < k) atomicAdd(S.cnt + j, 1);
  }
  __syncthreads();
  if (w == 0) {
    int run = 0;
    for (int base = 0; base < k; base += 32) {
      const int j = base + l;
      const int c = j < k ? S.cnt[j] : 0;
      int x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (l >= o) x += y;
      }
      if (j < k) { S.start[j] = run + x - c; S.cur[j] = run + x - c; }
      run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (l == 0) S.start[k] = run;
  }
  __syncthreads();
  for (int i0 = 0; i0 < nrows; i0 += kTccThreads) {
    const int i = i0 + threadIdx.x;
    int j = i < nrows ? S.lab[i] : k;
    if (j < 0 || j > k) j = k;
    const unsigned peers = __match_any_sync(0xffffffffu, j);
    const int rank = __popc(peers & ((1u << l) - 1u));
    if (j < k && rank == 0) S.wc[w * k + j] = __popc(peers);
    __syncthreads();
    if (j < k) {
      int pos = S.cur[j] + rank;
      for (int u = 0; u < w; ++u) pos += S.wc[u * k + j];
      S.order[pos] = i;
    }
    __syncthreads();
    for (int jj = threadIdx.x; jj < k; jj += blockDim.x) {
      int add = 0;
      for (int u = 0; u < kTccWarps; ++u) {
        add += S.wc[u * k + jj];
        S.wc[u * k + jj] = 0;
      }
      S.cur[jj] += add;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- sweeps
// Stages features [f0, f0 + fw) of own rows (and of the k centroid rows of C
// when with_c) into shared memory with 16-byte asynchronous copies, all in
// flight at once (many small bulk copies would queue in the copy engine).
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
               :: "r"(smem_u32(dst_smem)), "l"(src) : "memory");
}

__device__ void tcc_stage(const ChunkArgs& a, const TccS& S, int r0, int nrows, int f0,
                          int fw, bool with_c) {
  const int q4 = fw >> 2, ss4 = S.sstride >> 2, np4 = a.npad >> 2, f4 = f0 >> 2;
  const float4* P4 = reinterpret_cast<const float4*>(a.P) + (size_t)r0 * np4 + f4;
  const float4* C4 = reinterpret_cast<const float4*>(a.C) + f4;
  float4* sP4 = reinterpret_cast<float4*>(S.sP);
  float4* sC4 = reinterpret_cast<float4*>(S.sC);
  // thread -> (row offset, float4 column): q4 threads per row
  const int per = kTccThreads / q4, c = threadIdx.x % q4, r = threadIdx.x / q4;
  if (r < per) {
    for (int i = r; i < nrows; i += per) cp_async16(sP4 + i * ss4 + c, P4 + (size_t)i * np4 + c);
    if (with_c)
      for (int j = r; j < a.k; j += per) cp_async16(sC4 + j * ss4 + c, C4 + (size_t)j * np4 + c);
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  __syncthreads();
}

__device__ __forceinline__ bool tcc_multi(const TccS& S, int i) {
  return __popc(S.cmask[i * 4]) + __popc(S.cmask[i * 4 + 1]) + __popc(S.cmask[i * 4 + 2]) +
             __popc(S.cmask[i * 4 + 3]) > 1;
}

// Exact distances of single-candidate rows to their centroid (-> dmin) and,
// when update, this CTA's partial sums of (p - c_j) over the members of every
// live centroid j (ascending rows) and its member counts.
__device__ void tcc_sweep(const ChunkArgs& a, const TccS& S, int r0, int nrows, bool update) {
  const int k = a.k, n = a.n, npad = a.npad, fb = a.tc_fb, b = blockIdx.x, ss = S.sstride;
  float4* p4 = reinterpret_cast<float4*>(S.part4);
  for (int f0 = 0; f0 < npad; f0 += fb) {
    const int fw = min(fb, npad - f0);
    const bool last = f0 + fw >= npad;
    tcc_stage(a, S, r0, nrows, f0, fw, true);
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      const int j = S.lab[i];
      if (j < 0 || j >= k || tcc_multi(S, i)) continue;
      float4 acc = f0 == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : p4[i];
      const float4* xp = reinterpret_cast<const float4*>(S.sP + i * ss);
      const float4* cp = reinterpret_cast<const float4*>(S.sC + j * ss);
      for (int q = 0; q < (fw >> 2); ++q) {
        const float4 x = xp[q], c = cp[q];
        const float e0 = x.x - c.x, e1 = x.y - c.y, e2 = x.z - c.z, e3 = x.w - c.w;
        acc.x = fmaf(e0, e0, acc.x);
        acc.y = fmaf(e1, e1, acc.y);
        acc.z = fmaf(e2, e2, acc.z);
        acc.w = fmaf(e3, e3, acc.w);
      }
      if (last) S.dmin[i] = (acc.x + acc.y) + (acc.z + acc.w);
      else p4[i] = acc;
    }
    if (update) {
      // fw / 4 threads per group, four consecutive features each (one
      // float4); groups take centroids in turn.  Each feature's sum runs
      // over the members in ascending order.  Padding features sum to zero.
      const int q4 = fw >> 2, ng = kTccThreads / q4;
      const int g = threadIdx.x / q4, c4 = threadIdx.x - g * q4, f = f0 + 4 * c4;
      if (g < ng && f < n) {
        const int nl = S.lidx[k];
        for (int q = g; q < nl; q += ng) {
          const int j = S.lidx[q];
          const float4 c = *reinterpret_cast<const float4*>(S.sC + j * ss + 4 * c4);
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
          const int e1 = S.start[j + 1];
#pragma unroll 4
          for (int e = S.start[j]; e < e1; ++e) {
            const float4 v = *reinterpret_cast<const float4*>(S.sP + S.order[e] * ss + 4 * c4);
            sum.x += v.x - c.x;
            sum.y += v.y - c.y;
            sum.z += v.z - c.z;
            sum.w += v.w - c.w;
          }
          if (BM_GUARD(j >= 0 && j < k, &a.ctl->status))
            *reinterpret_cast<float4*>(a.part_sum + ((size_t)b * k + j) * npad + f) = sum;
        }
      }
    }
    __syncthreads();
  }
  if (update)
    for (int j = threadIdx.x; j < k; j += blockDim.x) a.part_cnt[(size_t)b * k + j] = S.cnt[j];
  // the staging region is the MMA ring of the next pass: order these
  // generic-proxy writes before its bulk copies
  fence_proxy_async_smem();
  __syncthreads();
}

// Exact distances of own rows to the nc candidate rows in S.cand -> dc[c][i].
__device__ void tcc_sweep_cands(const ChunkArgs& a, const TccS& S, int r0, int nrows, int nc) {
  const int npad = a.npad, fb = a.tc_fb, R = a.rows_per_cta, ss = S.sstride;
  float4* p4 = reinterpret_cast<float4*>(S.part4);
  for (int f0 = 0; f0 < npad; f0 += fb) {
    const int fw = min(fb, npad - f0);
    const bool last = f0 + fw >= npad;
    tcc_stage(a, S, r0, nrows, f0, fw, false);
    for (int e = threadIdx.x; e < nrows * nc; e += blockDim.x) {
      const int c = e / nrows, i = e - c * nrows;
      float4 acc = f0 == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : p4[c * R + i];
      const float4* xp = reinterpret_cast<const float4*>(S.sP + i * ss);
      const float4* cp = reinterpret_cast<const float4*>(S.cand + c * npad + f0);
      for (int q = 0; q < (fw >> 2); ++q) {
        const float4 x = xp[q], y = cp[q];
        const float e0 = x.x - y.x, e1 = x.y - y.y, e2 = x.z - y.z, e3 = x.w - y.w;
        acc.x = fmaf(e0, e0, acc.x);
        acc.y = fmaf(e1, e1, acc.y);
        acc.z = fmaf(e2, e2, acc.z);
        acc.w = fmaf(e3, e3, acc.w);
      }
      if (last) S.dc[c * R + i] = (acc.x + acc.y) + (acc.z + acc.w);
      else p4[c * R + i] = acc;
    }
    __syncthreads();
  }
  fence_proxy_async_smem();   // see tcc_sweep
  __syncthreads();
}

// One assignment of own rows: labels and exact distances (lab, dmin) and,
// when update, the update partials.
__device__ bool tcc_assign(const ChunkArgs& a, const TccS& S, int r0, int nrows,
                           const TccBound& bd, uint32_t tmem, TccPipe& pp, bool update,
                           uint64_t* tsub) {
  bool ok = tcc_pass_a(a, S, r0, nrows, bd, tmem, pp);
  phase_tick(a, 8, tsub);
  tcc_pass_multi(a, S, r0, nrows);
  if (update) tcc_sort(a, S, nrows);
  phase_tick(a, 9, tsub);
  tcc_sweep(a, S, r0, nrows, update);
  phase_tick(a, 10, tsub);
  return ok;
}

// ---------------------------------------------------------------- reduce
// New centroids from the partials, one warp per (centroid, 8-feature slice):
// the member count over CTAs and the slice's sums over CTAs (lane l sums the
// CTAs u = l, l + 32, ... in that order, then a fixed xor butterfly),
// c <- c + sum / count, the slice's planes and squared norm.  Centroids
// without members become degenerate (Sec. 3.3) unless the launch keeps them
// in place.
//
// A task's loads (the CTAs' partials, the old centroid value) land in
// registers first and are summed later, so a warp issues the loads of its
// first task before the objective's round trip and those of its next task
// before finishing the current one.
constexpr int kRedSlots = 5;   // CTAs u = l + 32 i, i < kRedSlots, held in registers

struct RedTask {
  int q;                       // (centroid, slice) index, or -1
  int cnt[kRedSlots];
  float4 x0[kRedSlots], x1[kRedSlots];
  float c;                     // lane l < 8: the old value of feature 8 sl + l
};

__device__ __forceinline__ RedTask tcc_reduce_load(const ChunkArgs& a, const TccS& S, int q) {
  const int k = a.k, npad = a.npad, G = gridDim.x, l = threadIdx.x & 31;
  const int nsl = (npad + 7) >> 3;
  RedTask t;
  t.q = -1;
  t.c = 0.f;
  if (q >= k * nsl) return t;
  const int j = q / nsl, sl = q - j * nsl;
  if (!S.live[j]) return t;
  t.q = q;
  const bool two = sl * 8 + 4 < npad;   // the slice's second float4 exists
#pragma unroll
  for (int i = 0; i < kRedSlots; ++i) {
    const int u = l + 32 * i;
    const bool on = u < G;
    t.cnt[i] = on ? __ldcg(a.part_cnt + (size_t)u * k + j) : 0;
    const float4* ps =
        reinterpret_cast<const float4*>(a.part_sum + ((size_t)u * k + j) * npad + sl * 8);
    t.x0[i] = on ? __ldcg(ps) : make_float4(0.f, 0.f, 0.f, 0.f);
    t.x1[i] = on && two ? __ldcg(ps + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int f = sl * 8 + l;
  if (l < 8 && f < a.n) t.c = __ldcg(a.C + (size_t)j * npad + f);
  return t;
}

__device__ __forceinline__ void tcc_reduce_finish(const ChunkArgs& a, const RedTask& t,
                                                  bool stop) {
  const int k = a.k, npad = a.npad, n = a.n, G = gridDim.x, l = threadIdx.x & 31;
  const int nsl = (npad + 7) >> 3;
  const int j = t.q / nsl, sl = t.q - j * nsl;
  const bool two = sl * 8 + 4 < npad;
  int cnt = 0;
  float v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = 0.f;
#pragma unroll
  for (int i = 0; i < kRedSlots; ++i) {
    cnt += t.cnt[i];
    v[0] += t.x0[i].x; v[1] += t.x0[i].y; v[2] += t.x0[i].z; v[3] += t.x0[i].w;
    v[4] += t.x1[i].x; v[5] += t.x1[i].y; v[6] += t.x1[i].z; v[7] += t.x1[i].w;
  }
  for (int u = l + 32 * kRedSlots; u < G; u += 32) {   // grids beyond 32 kRedSlots CTAs
    cnt += __ldcg(a.part_cnt + (size_t)u * k + j);
    const float4* ps =
        reinterpret_cast<const float4*>(a.part_sum + ((size_t)u * k + j) * npad + sl * 8);
    const float4 x0 = __ldcg(ps);
    const float4 x1 = two ? __ldcg(ps + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    v[0] += x0.x; v[1] += x0.y; v[2] += x0.z; v[3] += x0.w;
    v[4] += x1.x; v[5] += x1.y; v[6] += x1.z; v[7] += x1.w;
  }
  cnt = warp_sum_i32(cnt);
  if (cnt == 0) {   // degenerate, or kept in place (planes and norm unchanged)
    if (!a.empty_keep && sl == 0 && l == 0) a.mask[j] = 0;
    return;
  }
  if (stop) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
  float mine = 0.f;
#pragma unroll
  for (int e = 0; e < 8; ++e) if ((l & 7) == e) mine = v[e];
  const int f = sl * 8 + l;
  const bool on = l < 8 && f < n;
  float c = 0.f;
  if (on) {
    c = t.c + mine / (float)cnt;
    a.C[(size_t)j * npad + f] = c;
    put_cb(a, j, f, c);
  }
  float sq = on ? c * c : 0.f;
  sq += __shfl_xor_sync(0xffffffffu, sq, 1);
  sq += __shfl_xor_sync(0xffffffffu, sq, 2);
  sq += __shfl_xor_sync(0xffffffffu, sq, 4);
  if (l == 0) a.sqs[(size_t)j * nsl + sl] = sq;
}

// Every task of this warp, the first one's loads already issued (`first`).
__device__ void tcc_reduce(const ChunkArgs& a, const TccS& S, bool stop, const RedTask& first) {
  const int nsl = (a.npad + 7) >> 3, tasks = a.k * nsl;
  const int w = threadIdx.x >> 5;
  const int gw = blockIdx.x * kTccWarps + w, nw = gridDim.x * kTccWarps;
  RedTask cur = first;
  for (int q = gw; q < tasks; q += nw) {
    const RedTask nxt = tcc_reduce_load(a, S, q + nw);
    if (cur.q >= 0) tcc_reduce_finish(a, cur, stop);
    cur = nxt;
  }
  fence_proxy_async_global();   // the planes are read by bulk copies after the barrier
}

// ---------------------------------------------------------------- K-means++
// Centroid j <- row src (shared memory): CTA 0 publishes it (C, planes,
// norms, mask); every CTA marks it live.
__device__ void tcc_set_centroid(const ChunkArgs& a, const TccS& S, int j, const float* src) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nch = (a.npad + 31) >> 5;
  if (blockIdx.x == 0) {
    for (int ch = w; ch < nch; ch += kTccWarps) {
      const int f = ch * 32 + l;
      publish32(a, j, ch, f < a.npad ? src[f] : 0.f, true);
    }
    if (threadIdx.x == 0) a.mask[j] = 1;
    fence_proxy_async_global();
  }
  if (threadIdx.x == 0) S.live[j] = 1;
  __syncthreads();
}

__device__ __forceinline__ void tcc_load_cand(const ChunkArgs& a, const TccS& S, int c, int row) {
  if (!BM_GUARD(row >= 0 && row < a.s, &a.ctl->status)) row = 0;
  for (int f = threadIdx.x; f < a.npad; f += blockDim.x)
    S.cand[c * a.npad + f] = __ldcg(a.P + (size_t)row * a.npad + f);
}

// K-means++ reseed of every degenerate slot, ascending (Sec. 3.3, Sec. 5).
__device__ bool tcc_kpp(const ChunkArgs& a, const TccS& S, GridBarrier& gb, int r0, int nrows,
                        TccBound& bd, uint32_t tmem, TccPipe& pp, long long* nd_out,
                        uint64_t* tsub, unsigned long long gen) {
  const int k = a.k, G = gridDim.x, b = blockIdx.x, R = a.rows_per_cta;
  const int nlive = S.lidx[k];
  if (nlive == k) return true;
  if (a.init == kInitForgy) {
    // Forgy: slot j <- sample row floor(u_j * s), u_j its first K-means++
    // uniform; no distances, every CTA applies the same picks
    for (int j = 0; j < k; ++j) {
      if (S.live[j]) continue;
      const double u = unit_double(philox_word(a.seed, (uint64_t)a.t, 2, 0,
                                               (uint64_t)(j * a.trials)));
      tcc_load_cand(a, S, 0, min(a.s - 1, (int)floor(u * (double)a.s)));
      __syncthreads();
      tcc_set_centroid(a, S, j, S.cand);
    }
    build_live_list(S.live, S.lidx, k);
    if (!gb.sync()) return false;
    load_norms(a, S, &bd);
    return true;
  }
  long long nd = 0;
  double* DSUM = a.part_f + (size_t)kMaxTrials * G;
  bool ok = true;
  if (nlive > 0) {
    ok = tcc_assign(a, S, r0, nrows, bd, tmem, pp, false, tsub);
    nd += (long long)a.s * nlive;
  } else {
    const double uf = unit_double(philox_word(a.seed, (uint64_t)a.t, 1, 0, 0));
    const int i0 = (int)floor(uf * (double)a.s);
    tcc_load_cand(a, S, 0, i0);
    __syncthreads();
    tcc_set_centroid(a, S, 0, S.cand);
    tcc_sweep_cands(a, S, r0, nrows, 1);
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) S.dmin[i] = S.dc[i];
    __syncthreads();
    nd += a.s;
  }
  __shared__ int s_rows[kMaxTrials];
  for (int j = 0; j < k && ok; ++j) {
    if (S.live[j]) continue;
    const unsigned long long tag = kx_tag(gen, j);
    const double mine = dmin_sum(S.dmin, nrows, S.red);
    kpp_put_dsum(a, DSUM, mine, tag);
    if (!gb.sync()) { ok = false; break; }
    if (!kpp_locate(a, S.dmin, r0, nrows, DSUM, j, tag)) { ok = false; break; }
    if (!gb.sync()) { ok = false; break; }
    if (!kpp_get_cands(a, s_rows, tag)) { ok = false; break; }
    for (int t = 0; t < a.trials; ++t) tcc_load_cand(a, S, t, s_rows[t]);
    __syncthreads();
    tcc_sweep_cands(a, S, r0, nrows, a.trials);
    double pot[kMaxTrials];
    for (int t = 0; t < a.trials; ++t) {
      double v = 0.0;
      for (int i = threadIdx.x; i < nrows; i += blockDim.x)
        v += (double)fminf(S.dmin[i], S.dc[t * R + i]);
      pot[t] = block_sum_f64(v, S.red);
    }
    kpp_put_potentials(a, pot, tag);
    nd += (long long)a.s * a.trials;
    if (!gb.sync()) { ok = false; break; }
    const int bt = kpp_best(a, tag);
    if (bt < 0) { ok = false; break; }
    tcc_set_centroid(a, S, j, S.cand + bt * a.npad);
    for (int i = threadIdx.x; i < nrows; i += blockDim.x)
      S.dmin[i] = fminf(S.dmin[i], S.dc[bt * R + i]);
    __syncthreads();
  }
  build_live_list(S.live, S.lidx, k);
  // publish the reseeded rows (C, planes, norms) before Lloyd
  if (ok && !gb.sync()) ok = false;
  if (ok) load_norms(a, S, &bd);
  *nd_out += nd;
  return ok;
}

// ---------------------------------------------------------------- Lloyd
__device__ bool tcc_lloyd(const ChunkArgs& a, const TccS& S, GridBarrier& gb, int r0, int nrows,
                          TccBound& bd, uint32_t tmem, TccPipe& pp, long long* nd_out,
                          double* f_out, int* it_out, uint64_t* tclk) {
  const int k = a.k, G = gridDim.x, b = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  double* FPART = a.part_f + (size_t)(kMaxTrials + 1) * G;
  __shared__ double s_f;
  double f_prev = 0.0, f = 0.0;
  int it = 0;
  long long nd = 0;
  bool ok = true;
  while (true) {
    const int nlive = S.lidx[k];
    uint64_t tsub = *tclk;
    if (!tcc_assign(a, S, r0, nrows, bd, tmem, pp, true, &tsub)) ok = false;
    const double fp = dmin_sum(S.dmin, nrows, S.red);
    if (threadIdx.x == 0) FPART[b] = fp;
    nd += (long long)a.s * nlive;
    phase_tick(a, 3, tclk);
    if (!ok || !gb.sync()) { ok = false; break; }
    phase_tick(a, 4, tclk);
    const RedTask first = tcc_reduce_load(a, S, b * kTccWarps + w);
    if (w == 0) {
      const double t = warp_sum_array_f64(FPART, G);
      if (l == 0) s_f = t;
    }
    __syncthreads();
    f = s_f;
    const bool stop = (f == 0.0) || (it > 0 && f_prev - f <= a.tol * f_prev) ||
                      (it == a.max_iter);
    tcc_reduce(a, S, stop, first);
    phase_tick(a, 5, tclk);
    if (!gb.sync()) { ok = false; break; }
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      S.live[j] = __ldcg(reinterpret_cast<const unsigned char*>(a.mask) + j) != 0;
    build_live_list(S.live, S.lidx, k);
    if (!stop) load_norms(a, S, &bd);
    phase_tick(a, 6, tclk);
    if (stop) break;
    f_prev = f;
    ++it;
  }
  *nd_out += nd;
  *f_out = f;
  *it_out = it;
  return ok;
}

// ---------------------------------------------------------------- gather
// P[i] = X[idx[i]] for own rows (zero padding to npad).  Rows of X that are
// 16-byte aligned move as float4 (eight loads in flight per thread), others
// as 32-feature units (sixteen in flight per warp).
__device__ void tcc_gather(const ChunkArgs& a, const TccS& S, int r0, int nrows) {
  const int n = a.n, npad = a.npad, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) S.order[i] = __ldcg(a.idx + r0 + i);
  __syncthreads();
  const long long ready = gather_rows_ready(a, r0, nrows);
  if ((n & 3) == 0 && gather_sources_aligned16(a)) {
    const int q4 = npad >> 2, units = nrows * q4;
    float4* P4 = reinterpret_cast<float4*>(a.P) + (size_t)r0 * q4;
    for (int u0 = threadIdx.x; u0 < units; u0 += 8 * kTccThreads) {
      float4 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int u = u0 + q * kTccThreads;
        if (u < units) {
          const int i = u / q4, c = u - i * q4;
          int row = S.order[i];
          if (!BM_GUARD(row >= 0 && row < a.m, &a.ctl->status)) row = 0;
          v[q] = __ldg(reinterpret_cast<const float4*>(gather_row_source(a, row, ready)) +
                       (size_t)row * q4 + c);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int u = u0 + q * kTccThreads;
        if (u < units) P4[u] = v[q];
      }
    }
  } else {
    const int nch = (npad + 31) >> 5;
    const int units = nrows * nch;
    for (int u0 = w * 16; u0 < units; u0 += 16 * kTccWarps) {
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int u = u0 + q;
        v[q] = 0.f;
        if (u < units) {
          const int i = u / nch, f = (u - i * nch) * 32 + l;
          const int row = S.order[i];
          if (f < n && BM_GUARD(row >= 0 && row < a.m, &a.ctl->status))
            v[q] = __ldg(gather_row_source(a, row, ready) + (size_t)row * n + f);
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int u = u0 + q;
        if (u < units) {
          const int i = u / nch, f = (u - i * nch) * 32 + l;
          if (f < npad) a.P[(size_t)(r0 + i) * npad + f] = v[q];
        }
      }
    }
  }
  __syncthreads();
}

// Whether the gather can build the BF16 row tiles itself (tcc_gather_convert):
// rows of 16-byte units from 16-byte aligned sources, whole 8-feature chunks,
// and at most 16 K blocks (the norm partials' scratch).
__device__ __forceinline__ bool tcc_fused_gather_ok(const ChunkArgs& a) {
  return !a.tc_fp8 && (a.n & 3) == 0 && (a.npad & 7) == 0 && a.tc_kb <= 16 &&
         gather_sources_aligned16(a);
}

// tcc_gather and tcc_convert_own in one pass: every 8-feature chunk of an
// own row goes from X to registers once and from there to P (FP32), to the
// row tiles (BF16 planes, the same bits as tcc_convert_own) and to the
// chunk's share of the row norm.  Units are (tile row, 8-feature chunk) over
// whole tiles and K blocks, so the eight lanes of a (row, K block) are
// consecutive and the padding rows and features of the tiles are written as
// zeros, as tcc_convert_own writes them.  Each thread keeps kGcUnits units
// (16 float4 loads) in flight.  The norm of row i adds its K blocks' sums in
// block order into 0, as tcc_convert_own does, through per-(row, block)
// partials in the part4 scratch.
constexpr int kGcUnits = 8;
__device__ void tcc_gather_convert(const ChunkArgs& a, const TccS& S, int r0, int nrows) {
  const int tid = threadIdx.x, kb = a.tc_kb, npad = a.npad;
  const int cpr = kb * 8;                                  // 8-feature chunks per tile row
  const int ntl = (nrows + kTccM - 1) / kTccM;
  const int units = ntl * kTccM * cpr;
  const int blk = a.tc_planes * kTccM * 128;
  float* nqs = reinterpret_cast<float*>(S.part4);          // [nrows][kb] norm partials
  for (int i = tid; i < nrows; i += blockDim.x) S.order[i] = __ldcg(a.idx + r0 + i);
  __syncthreads();
  const long long ready = gather_rows_ready(a, r0, nrows);
  unsigned char* base = a.Pb + (size_t)blockIdx.x * a.tc_tpc * kb * blk;
  // the trip count depends on the units only, so every lane reaches the
  // shuffles below
  for (int u0 = 0; u0 < units; u0 += kGcUnits * kTccThreads) {
    float4 v[kGcUnits][2];
#pragma unroll
    for (int q = 0; q < kGcUnits; ++q) {
      const int u = u0 + q * kTccThreads + tid;
      const int i = u / cpr, f0 = (u - i * cpr) * 8;
      v[q][0] = v[q][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (u < units && i < nrows && f0 < npad) {
        int row = S.order[i];
        if (!BM_GUARD(row >= 0 && row < a.m, &a.ctl->status)) row = 0;
        const float4* src = reinterpret_cast<const float4*>(
            gather_row_source(a, row, ready) + (size_t)row * a.n + f0);
        v[q][0] = __ldg(src);
        v[q][1] = __ldg(src + 1);
      }
    }
#pragma unroll
    for (int q = 0; q < kGcUnits; ++q) {
      const int u = u0 + q * kTccThreads + tid;
      const int i = u / cpr, c8 = u - i * cpr, f0 = c8 * 8;
      const bool real = u < units && i < nrows && f0 < npad;
      if (real) {
        float4* dstp = reinterpret_cast<float4*>(a.P + (size_t)(r0 + i) * npad + f0);
        dstp[0] = v[q][0];
        dstp[1] = v[q][1];
      }
      const float x[8] = {v[q][0].x, v[q][0].y, v[q][0].z, v[q][0].w,
                          v[q][1].x, v[q][1].y, v[q][1].z, v[q][1].w};
      float nq = 0.f;
      uint32_t h[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        nq = fmaf(x[2 * e], x[2 * e], nq);
        nq = fmaf(x[2 * e + 1], x[2 * e + 1], nq);
        const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(x[2 * e] - hf.x, x[2 * e + 1] - hf.y);
        h[e] = *reinterpret_cast<const uint32_t*>(&hh);
        lo[e] = *reinterpret_cast<const uint32_t*>(&ll);
      }
      if (u < units) {
        const int b = c8 >> 3, ch = c8 & 7, tl = i / kTccM, r = i - tl * kTccM;
        unsigned char* dst = base + (size_t)(tl * kb + b) * blk;
        const int off = sw128_offset(r, ch * 8);
        *reinterpret_cast<uint4*>(dst + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (a.tc_planes == 2)
          *reinterpret_cast<uint4*>(dst + kTccM * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      // the eight lanes of a (row, K block) are consecutive
      nq += __shfl_xor_sync(0xffffffffu, nq, 1);
      nq += __shfl_xor_sync(0xffffffffu, nq, 2);
      nq += __shfl_xor_sync(0xffffffffu, nq, 4);
      if ((c8 & 7) == 0 && u < units && i < nrows) nqs[i * kb + (c8 >> 3)] = nq;
    }
  }
  fence_proxy_async_global();   // the tiles are read back by bulk copies
  __syncthreads();
  for (int i = tid; i < nrows; i += blockDim.x) {
    float xx = 0.f;
    for (int b = 0; b < kb; ++b) xx += nqs[i * kb + b];
    S.xx[i] = xx;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- incumbent
// The (centroid, 32-feature unit) pairs of C' <- C that CTA b publishes:
// q = b * warps + w, then every gridDim.x * warps.
__device__ void tcc_publish_incumbent(const ChunkArgs& a, const TccS& S, const float* src,
                                      bool full) {
  const int k = a.k, nch = (a.npad + 31) >> 5;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int q = blockIdx.x * kTccWarps + w; q < k * nch; q += gridDim.x * kTccWarps) {
    const int j = q / nch, ch = q - j * nch, f = ch * 32 + l;
    const float v = f < a.npad ? __ldcg(src + (size_t)j * a.npad + f) : 0.f;
    publish32(a, j, ch, v, full);
  }
  if (full && blockIdx.x == 0)
    for (int j = threadIdx.x; j < k; j += blockDim.x) a.mask[j] = S.live[j];
  fence_proxy_async_global();
}

// Largest magnitude over the live incumbent values of those same pairs
// (every thread gets it).
__device__ float tcc_incumbent_max(const ChunkArgs& a, const TccS& S, const float* src) {
  const int k = a.k, nch = (a.npad + 31) >> 5;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float m = 0.f;
  for (int q = blockIdx.x * kTccWarps + w; q < k * nch; q += gridDim.x * kTccWarps) {
    const int j = q / nch, f = (q - j * nch) * 32 + l;
    if (S.live[j] && f < a.n) m = fmaxf(m, fabsf(__ldcg(src + (size_t)j * a.npad + f)));
  }
  m = warp_max_f32(m);
  __syncthreads();
  if (l == 0) S.red[w] = m;
  __syncthreads();
  float all = 0.f;
  for (int i = 0; i < kTccWarps; ++i) all = fmaxf(all, (float)S.red[i]);
  __syncthreads();
  return all;
}

// E4M3 centroid scale of the chunk from the CTAs' shares of M (after the
// grid barrier): cs = 2^(7 - floor(log2 M)), so M cs lies in [128, 256).
__device__ void tcc_set_cscale(const double* mpart) {
  if (threadIdx.x < 32) {
    float m = 0.f;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) m = fmaxf(m, (float)__ldcg(mpart + i));
    m = warp_max_f32(m);
    if (threadIdx.x == 0) {
      const int e2 = (m > 0.f && m <= 3.0e38f) ? max(ilogbf(m), -119) : 7;
      fp8_cscale()[0] = ldexpf(1.f, 7 - e2);
      fp8_cscale()[1] = ldexpf(1.f, e2 - 7);
      fp8_cscale()[2] = m;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- kernel
__global__ void __launch_bounds__(kTccThreads, 1) chunk_tc_kernel(ChunkArgs a) {
  extern __shared__ __align__(1024) unsigned char tcc_raw[];
  BM_POISON_SMEM();
  BM_START_SKEW();
  unsigned char* base = tcc_raw + ((1024u - (smem_u32(tcc_raw) & 1023u)) & 1023u);
  const int R = a.rows_per_cta, k = a.k;
  const TccLayout L = tcc_layout(a.npad, k, R, a.tc_n16, a.tc_fb, a.tc_ns, a.tc_planes);
  TccS S;
  S.ring = base + L.region;
  S.sP = reinterpret_cast<float*>(base + L.region);
  S.sC = reinterpret_cast<float*>(base + L.region + L.stage_c);
  S.cmask = reinterpret_cast<uint32_t*>(base + L.cmask);
  S.lab = reinterpret_cast<int*>(base + L.lab);
  S.dmin = reinterpret_cast<float*>(base + L.dmin);
  S.part4 = reinterpret_cast<float*>(base + L.part4);
  S.dc = reinterpret_cast<float*>(base + L.dc);
  S.order = reinterpret_cast<int*>(base + L.order);
  S.cnt = reinterpret_cast<int*>(base + L.cnt);
  S.start = reinterpret_cast<int*>(base + L.start);
  S.cur = reinterpret_cast<int*>(base + L.cur);
  S.wc = reinterpret_cast<int*>(base + L.wc);
  S.cand = reinterpret_cast<float*>(base + L.cand);
  S.live = reinterpret_cast<int*>(base + L.live);
  S.lidx = reinterpret_cast<int*>(base + L.lidx);
  S.cc = reinterpret_cast<float*>(base + L.cc);
  S.xx = reinterpret_cast<float*>(base + L.xx);
  S.rsc = reinterpret_cast<float*>(base + L.rsc);
  S.xm = reinterpret_cast<float*>(base + L.xm);
  S.mlist = reinterpret_cast<int*>(base + L.mlist);
  S.red = reinterpret_cast<double*>(base + L.red);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bars);
  S.bfull = bars;
  S.sfree = bars + 3;
  S.accb = bars + 6;
  S.holder = reinterpret_cast<uint32_t*>(base + L.holder);
  S.sstride = L.sstride;
  S.ring_slot = L.ring_slot;
  S.ring_a = L.ring_a;
  S.ns = a.tc_ns;

  GridBarrier gb{a.ctl->bar + a.bar_sel, &a.ctl->status, 0u};
  const unsigned long long gen = kx_generation(a);
  const int r0 = min(a.s, (int)blockIdx.x * R);
  const int nrows = min(R, a.s - r0);
  long long nd = 0;
  double f = 0.0;
  int it = 0;
  bool ok = true;
  TccPipe pp{0u, 0u};
  TccBound bd{0.f, 0.f};

  if (threadIdx.x < kNumPhaseTimers) phase_slots()[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 7; ++i) mbar_init(bars + i, 1);
    mbar_init_fence();
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(S.holder, (uint32_t)a.tc_ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *S.holder;
  uint64_t tclk = trace_now(a);

  const bool full = (a.phases & kPhaseKeep) != 0;
  const bool work = (a.phases & (kPhaseKpp | kPhaseLloyd)) != 0;
  const float* csrc = full ? a.Cinc : a.C;
  if (work) {
    // C' <- C (Alg. 1): the working copy starts from the incumbent; its
    // planes and slice norms are rebuilt by all CTAs together (E4M3: once
    // the chunk's centroid scale is known, below)
    const uint8_t* msrc = full ? a.mask_inc : a.mask;
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      S.live[j] = __ldcg(reinterpret_cast<const unsigned char*>(msrc) + j) != 0;
    build_live_list(S.live, S.lidx, k);
    if (!a.tc_fp8) tcc_publish_incumbent(a, S, csrc, full);
  }
  phase_tick(a, 0, &tclk);
  // BF16 forms: the gather builds the row tiles as it goes
  const bool fused = work && (a.phases & kPhaseGather) && tcc_fused_gather_ok(a);
  if (fused) tcc_gather_convert(a, S, r0, nrows);
  else if (a.phases & kPhaseGather) tcc_gather(a, S, r0, nrows);
  if (work && a.tc_fp8) {
    // M = the largest magnitude over the sample rows and the live incumbent
    // centroids: each CTA's share (own rows, the incumbent values it
    // publishes), exchanged through one grid barrier
    double* MPART = a.part_f + (size_t)(kMaxTrials + 1) * gridDim.x;
    const float mine = fmaxf(tcc_convert_own_fp8(a, S, r0, nrows), tcc_incumbent_max(a, S, csrc));
    if (threadIdx.x == 0) MPART[blockIdx.x] = (double)mine;
    ok = gb.sync();
    if (ok) {
      tcc_set_cscale(MPART);
      tcc_publish_incumbent(a, S, csrc, full);
    }
  } else if (work && !fused) {
    tcc_convert_own(a, S, r0, nrows);
  }
  if (work) {
    ok = ok && gb.sync();
    if (ok) load_norms(a, S, &bd);
  }
  phase_tick(a, 1, &tclk);
  if (ok && (a.phases & kPhaseKpp)) {
    uint64_t tsub = tclk;
    ok = tcc_kpp(a, S, gb, r0, nrows, bd, tmem, pp, &nd, &tsub, gen);
    phase_tick(a, 2, &tclk);
  }
  if (ok && (a.phases & kPhaseLloyd))
    ok = tcc_lloyd(a, S, gb, r0, nrows, bd, tmem, pp, &nd, &f, &it, &tclk);
  if (ok && blockIdx.x == 0) {
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
      for (int q = threadIdx.x; q < k * a.npad; q += blockDim.x) a.Cinc[q] = __ldcg(a.C + q);
      for (int j = threadIdx.x; j < k; j += blockDim.x)
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
  // release TMEM on every path (the MMAs have completed: every pass waits
  // for its accumulator)
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, (uint32_t)a.tc_ncols);
}

// ---------------------------------------------------------------- host side
size_t chunk_tc_smem(int npad, int k, int R, int n16, int fb, int ns, int planes) {
  const TccLayout L = tcc_layout(npad, k, R, n16, fb, ns, planes);
  return (size_t)L.total + 1024;   // + alignment slack of the dynamic base
}

int chunk_tc_max_grid(size_t smem) {
  if (allow_max_smem(chunk_tc_kernel) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chunk_tc_kernel, kTccThreads,
                                                    smem) != cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::min(per_sm, 1) * sms;   // one CTA per SM: TMEM and the grid barrier
}

cudaError_t launch_chunk_tc(const ChunkArgs& a, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_max_smem(chunk_tc_kernel);
  if (e != cudaSuccess) return e;
  return launch_cooperative(chunk_tc_kernel, grid, kTccThreads, smem, st, a);
}

}  // namespace bm
