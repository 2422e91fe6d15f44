// Streaming tensor-core final assignment (Alg. 1's last step, Sec. 3.4) for
// rows of at most 128 features: the same distances, error bound, candidate
// rule and exact FP32 rescoring as assign_tc_kernel (bm_tc.cu), organised
// for HBM rate.
//
// One persistent CTA per SM with these roles:
//   - a TMA warp streams the CTA's 128-row tiles of X into a ring of
//     shared-memory stages, one 128-byte-wide column box (32 features x 128
//     rows, 128-byte swizzle) per stage;
//   - W compute warpgroups (two, or four for rows of at most 32 features,
//     whose registers allow it) take tiles in turn.  Each thread owns one row:
//     it copies the row's boxes from the stages into registers (the swizzle
//     makes these reads conflict-free) and releases the stages at once, writes
//     the BF16 (hi[, lo]) operand of the row into the shared A tile and the
//     row norm; after the MMA it reads the row's approximate distances from
//     TMEM, keeps the candidates, and rescores them exactly from the row in
//     its registers and the FP32 centroids in shared memory;
//   - an MMA warp issues the tile's tcgen05.mma (FP32 accumulators in one of
//     W TMEM buffers, so one warpgroup's epilogue overlaps the others'
//     conversion and MMA).  The A tile has NA buffers: one per warpgroup
//     where shared memory allows, so conversions do not wait for each
//     other's MMAs, else one shared buffer.
// The FP32 row never goes back to memory after its first read, so stages
// turn over as fast as HBM fills them.
#include <algorithm>
#include <climits>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "bm_device.cuh"
#include "bm_internal.h"
#include "bm_tc.cuh"

namespace bm {

constexpr int kTcsRows = 128;
constexpr int kTcsBox = 32 * 128 * 4;             // one stage: 32 features x 128 rows FP32
constexpr int kTcsMaxStages = 8;
constexpr int kTcsMaxW = 4;
// W compute warpgroups + the TMA warp + the MMA warp
__host__ __device__ constexpr int tcs_threads(int W) { return W * 128 + 64; }

struct TcsLayout {
  int sA, sB, stg, cF, cc, bars, holder, pair, total;
};

__host__ __device__ inline TcsLayout tcs_layout(int nb, int N, int k, int planes, int stages,
                                                int na) {
  const int kb = (nb * 32 + 63) / 64;
  TcsLayout L;
  int o = 0;
  L.sA = o;    o += na * planes * kb * kTcsRows * 128;  // A tiles, BF16 swizzled
  L.sB = o;    o += planes * kb * N * 128;              // centroids, BF16 swizzled
  L.stg = o;   o += stages * kTcsBox;                   // FP32 column boxes (TMA)
  L.cF = o;    o += align_up(k * (nb * 32 + 4) * 4, 16);   // FP32 centroids, padded rows
  L.cc = o;    o += align_up(N * 4, 16);                // ||c_j||^2, +inf if not live
  L.bars = o;  o += (2 * kTcsMaxStages + 3 * kTcsMaxW) * 8;
  L.holder = o; o += 16;
  L.pair = o;  o += 4 * kTcsMaxW * 8;                   // per-warp SSE pairs
  L.total = o;
  return L;
}

struct TcsArgs {
  long long m;
  int n, k, N, terms, stages, ncols;
  const float* C;
  int cstride;
  const uint8_t* mask;
  int32_t* labels;
  float* dmin;
  float2* part;
  double* sse;
  uint32_t* ticket;
  unsigned long long* rescored;
  int* status;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(mbar)) : "memory");
}

// TMA: box (x, y) of the 2-D tensor map -> shared memory, completing the
// box's bytes on the mbarrier.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
         "r"(smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void wg_sync(int wg) {
  asm volatile("bar.sync %0, 128;" :: "r"(1 + wg) : "memory");
}

// W = 2: 320 threads leave 168 registers a thread (rows of up to 96
// features stay in registers, 128-feature rows spill a few values); W = 4:
// 576 threads, rows of up to 32 features.
template <int NB, int W, int NA>
__global__ void __launch_bounds__(tcs_threads(W), 1)
assign_tcs_kernel(const __grid_constant__ CUtensorMap xmap, TcsArgs a) {
  constexpr int kThreads = tcs_threads(W);
  extern __shared__ __align__(1024) unsigned char tcs_raw[];
  BM_POISON_SMEM();
  unsigned char* sm = tcs_raw + ((1024u - (smem_u32(tcs_raw) & 1023u)) & 1023u);
  constexpr int NF = NB * 32;                // features held per row (zero padded)
  constexpr int KB = (NF + 63) / 64;         // K blocks of 64 BF16
  constexpr int CS = NF + 4;                 // cF row stride (floats)
  const int n = a.n, k = a.k, N = a.N, S = a.stages;
  const int planes = a.terms == 3 ? 2 : 1;
  const TcsLayout L = tcs_layout(NB, N, k, planes, S, NA);
  unsigned char* sA = sm + L.sA;
  unsigned char* sB = sm + L.sB;
  float* stg = reinterpret_cast<float*>(sm + L.stg);
  float* cF = reinterpret_cast<float*>(sm + L.cF);
  float* cc = reinterpret_cast<float*>(sm + L.cc);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* empty = full + kTcsMaxStages;
  uint64_t* sa_full = empty + kTcsMaxStages;   // [NA]
  uint64_t* mma_done = sa_full + kTcsMaxW;     // [W]
  uint64_t* tmem_free = mma_done + kTcsMaxW;   // [W]
  uint32_t* holder = reinterpret_cast<uint32_t*>(sm + L.holder);
  float2* pair = reinterpret_cast<float2*>(sm + L.pair);
  __shared__ float s_bound[2];
  __shared__ float s_cmax[kThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ntiles = (a.m + kTcsRows - 1) / kTcsRows;
  const int planeA = KB * kTcsRows * 128, planeB = KB * N * 128;
  const int bufA = planes * planeA;   // bytes of one A buffer

  // ---- set-up: zero A (its K padding stays zero), build B, cF, cc
  for (int q = tid; q < NA * bufA / 16; q += kThreads)
    reinterpret_cast<uint4*>(sA)[q] = make_uint4(0u, 0u, 0u, 0u);
  for (int e = tid; e < N * KB * 64; e += kThreads) {
    const int j = e / (KB * 64), f = e - j * (KB * 64);
    float v = 0.f;
    if (j < k && f < n && a.mask[j]) v = __ldg(a.C + (size_t)j * a.cstride + f);
    if (j < k && f < CS) cF[j * CS + f] = v;
    const int off = (f >> 6) * N * 128 + sw128_offset(j, f & 63);
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(sB + off) = h;
    if (planes == 2)
      *reinterpret_cast<__nv_bfloat16*>(sB + planeB + off) =
          __float2bfloat16_rn(v - __bfloat162float(h));
  }
  for (int e = tid; e < k * 4; e += kThreads)   // cF pad columns NF .. NF + 3
    if (KB * 64 < CS) cF[(e >> 2) * CS + KB * 64 + (e & 3)] = 0.f;
  float cmax = 0.f;
  for (int j = tid; j < N; j += kThreads) {
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
  const float eps = planes == 1 ? 1.01f * 0x1.0p-7f + (float)(n + 16) * 0x1.0p-22f
                                : 3.1f * 0x1.0p-16f + (float)(3 * n + 16) * 0x1.0p-22f;
  cmax = warp_max_f32(cmax);
  if (lane == 0) s_cmax[warp] = cmax;
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 128);
    }
    for (int i = 0; i < NA; ++i) mbar_init(sa_full + i, 128);
    for (int i = 0; i < W; ++i) {
      mbar_init(mma_done + i, 1);
      mbar_init(tmem_free + i, 128);
    }
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(holder, (uint32_t)a.ncols);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    float mx = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, s_cmax[w]);
    s_bound[0] = 2.f * eps * sqrtf(mx) * 1.0001f;
    s_bound[1] = (float)(n + 2) * 0x1.0p-22f * mx;
  }
  __syncthreads();
  const uint32_t tmem = *holder;
  bool ok = true;

  if (warp == 4 * W) {
    // ---- TMA producer: boxes in (tile, box) order through the ring
    if (lane == 0) {
      long long seq = 0;
      for (long long li = 0;; ++li) {
        const long long t = (long long)blockIdx.x + li * gridDim.x;
        if (t >= ntiles) break;
        for (int b = 0; b < NB; ++b, ++seq) {
          const int slot = (int)(seq % S);
          if (seq >= S && !mbar_wait(empty + slot, (uint32_t)(((seq / S) - 1) & 1))) ok = false;
          mbar_expect_tx(full + slot, (uint32_t)kTcsBox);
          tma_load_2d(stg + (size_t)slot * (kTcsBox / 4), &xmap, b * 32, (int)(t * kTcsRows),
                      full + slot);
        }
      }
      // no copy may still be landing when the CTA exits: the last boxes of
      // every slot have normally been consumed already
      for (long long q = seq - 1; q >= 0 && q >= seq - S; --q)
        if (!mbar_wait(full + (int)(q % S), (uint32_t)((q / S) & 1))) ok = false;
    }
  } else if (warp == 4 * W + 1) {
    // ---- MMA issuer: tile li from A buffer li % NA into TMEM buffer li % W
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(kTcsRows, N);
      const uint64_t da = sdesc_sw128(smem_u32(sA));
      const uint64_t db = sdesc_sw128(smem_u32(sB));
      const uint64_t alo = (uint64_t)(planeA >> 4), blo = (uint64_t)(planeB >> 4);
      for (long long li = 0;; ++li) {
        const long long t = (long long)blockIdx.x + li * gridDim.x;
        if (t >= ntiles) break;
        if (!mbar_wait(sa_full + (li % NA), (uint32_t)((li / NA) & 1))) ok = false;
        if (li >= W && !mbar_wait(tmem_free + (li % W), (uint32_t)(((li - W) / W) & 1)))
          ok = false;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)((li % W) * N);
        const uint64_t dab = da + (uint64_t)(((li % NA) * bufA) >> 4);
        uint32_t acc = 0;
        for (int b = 0; b < KB; ++b)
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t off = (uint64_t)((ks * 32) >> 4);
            const uint64_t ab = dab + (uint64_t)((b * kTcsRows * 128) >> 4) + off;
            const uint64_t bb = db + (uint64_t)((b * N * 128) >> 4) + off;
            tc_mma_bf16(d, ab, bb, idesc, acc);                 // hi * hi
            acc = 1;
            if (planes == 2) {
              tc_mma_bf16(d, ab, bb + blo, idesc, 1);           // hi * lo
              tc_mma_bf16(d, ab + alo, bb, idesc, 1);           // lo * hi
            }
          }
        tc_commit(mma_done + (li % W));
      }
    }
  } else {
    // ---- compute warpgroups: warpgroup wg takes local tiles wg, wg + W, ...
    const int wg = warp >> 2, r = tid & 127, q = warp & 3;
    const float e_d = (float)(n + 4) * 0x1.0p-22f;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    unsigned rescored = 0;
    for (long long li = wg;; li += W) {
      const long long t = (long long)blockIdx.x + li * gridDim.x;
      if (t >= ntiles) break;
      const long long row = t * kTcsRows + r;
      const bool valid = row < a.m;
      // A buffer li % NA is free once the MMA of its previous tile, li - NA,
      // has completed
      if (li >= NA &&
          !mbar_wait(mma_done + ((li - NA) % W), (uint32_t)(((li - NA) / W) & 1)))
        ok = false;
      unsigned char* sAb = sA + (li % NA) * bufA;
      float x[NF];
      float xq = 0.f;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const long long seq = li * NB + b;
        const int slot = (int)(seq % S);
        if (!mbar_wait(full + slot, (uint32_t)((seq / S) & 1))) ok = false;
        const unsigned char* box = reinterpret_cast<const unsigned char*>(stg) +
                                   (size_t)slot * kTcsBox + r * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(box + ((c ^ (r & 7)) << 4));
          x[b * 32 + 4 * c] = v.x;
          x[b * 32 + 4 * c + 1] = v.y;
          x[b * 32 + 4 * c + 2] = v.z;
          x[b * 32 + 4 * c + 3] = v.w;
        }
        mbar_arrive(empty + slot);
        // BF16 operand chunks of this box: features b*32 .. b*32+31 are
        // chunks 4*(b&1) .. 4*(b&1)+3 of K block b/2
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t h[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float v0 = x[b * 32 + 8 * c + 2 * u], v1 = x[b * 32 + 8 * c + 2 * u + 1];
            xq = fmaf(v0, v0, xq);
            xq = fmaf(v1, v1, xq);
            const __nv_bfloat162 hh = __floats2bfloat162_rn(v0, v1);
            h[u] = *reinterpret_cast<const uint32_t*>(&hh);
            if (planes == 2) {
              const float2 hf = __bfloat1622float2(hh);
              const __nv_bfloat162 ll = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
              lo[u] = *reinterpret_cast<const uint32_t*>(&ll);
            }
          }
          const int ch = 4 * (b & 1) + c;
          const int off = (b >> 1) * (kTcsRows * 128) + (r >> 3) * 1024 + (r & 7) * 128 +
                          ((ch ^ (r & 7)) << 4);
          *reinterpret_cast<uint4*>(sAb + off) = make_uint4(h[0], h[1], h[2], h[3]);
          if (planes == 2)
            *reinterpret_cast<uint4*>(sAb + planeA + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(sa_full + (li % NA));
      if (!mbar_wait(mma_done + (li % W), (uint32_t)((li / W) & 1))) ok = false;
      tc_fence_after();

      // ---- epilogue: candidates from the approximate distances, exact rescoring
      const uint32_t cols = lane_base + (uint32_t)((li % W) * N);
      const float xqb = xq * 1.00002f;
      const float E1 = fmaf(sqrtf(xqb), s_bound[0], s_bound[1]);
      float m1 = INFINITY;
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(cols + (uint32_t)c0, v);
#pragma unroll
        for (int u = 0; u < 16; ++u) m1 = fminf(m1, fmaf(-2.f, v[u], cc[c0 + u]));
      }
      const float thr = m1 + 2.f * E1 + 3.f * e_d * fmaxf(0.f, xqb + m1 + E1);
      // every candidate of the row first (one mask over all N <= 128
      // columns), so that a warp's rescoring loop runs as often as its row
      // with the most candidates needs, not once per column chunk
      uint64_t mlo = 0ull, mhi = 0ull;
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(cols + (uint32_t)c0, v);
        uint32_t bits = 0u;
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (c0 + u < k && fmaf(-2.f, v[u], cc[c0 + u]) <= thr) bits |= 1u << u;
        if (c0 < 64) mlo |= (uint64_t)bits << c0;
        else mhi |= (uint64_t)bits << (c0 - 64);
      }
      tc_fence_before();
      mbar_arrive(tmem_free + (li % W));   // TMEM buffer free for tile li + W
      if (!valid) mlo = mhi = 0ull;
      float best = INFINITY;
      int bj = INT_MAX, ncand = 0;
      while (mlo | mhi) {   // ascending index
        int j;
        if (mlo) {
          j = __ffsll((long long)mlo) - 1;
          mlo &= mlo - 1ull;
        } else {
          j = 64 + __ffsll((long long)mhi) - 1;
          mhi &= mhi - 1ull;
        }
        ++ncand;
        // exact FP32 distance: four partial sums over f mod 4, the order of
        // the FP32 kernels (the zero padding adds exact zeros)
        const float4* c4 = reinterpret_cast<const float4*>(cF + j * CS);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int u = 0; u < NF / 4; ++u) {
          const float4 cv = c4[u];
          const float e0 = x[4 * u] - cv.x, e1 = x[4 * u + 1] - cv.y;
          const float e2 = x[4 * u + 2] - cv.z, e3 = x[4 * u + 3] - cv.w;
          s0 = fmaf(e0, e0, s0);
          s1 = fmaf(e1, e1, s1);
          s2 = fmaf(e2, e2, s2);
          s3 = fmaf(e3, e3, s3);
        }
        const float dd = (s0 + s1) + (s2 + s3);
        if (bj == INT_MAX || dd < best) { best = dd; bj = j; }
      }
      float th = valid ? best : 0.f, tl = 0.f;
      if (valid) {
        if (BM_GUARD(row < a.m && (bj == INT_MAX || bj < k), a.status)) {
          if (a.labels) a.labels[row] = bj;
          if (a.dmin) a.dmin[row] = best;
        }
        rescored += ncand > 1;
      }
      // the tile's SSE as an exact (hi, lo) pair: warps of the warpgroup,
      // then in warp order
      warp_two_sum(th, tl);
      if (lane == 0) pair[warp] = make_float2(th, tl);
      wg_sync(wg);
      if (r == 0) {
        float2 p = pair[wg * 4];
        for (int w = 1; w < 4; ++w) {
          two_sum_acc(p.x, p.y, pair[wg * 4 + w].x);
          p.y = __fadd_rn(p.y, pair[wg * 4 + w].y);
        }
        a.part[t] = p;
      }
      wg_sync(wg);
    }
    const unsigned resc = __reduce_add_sync(0xffffffffu, rescored);
    if (lane == 0 && resc) atomicAdd(a.rescored, (unsigned long long)resc);
  }
  if (!ok) atomicCAS(a.status, 0, kStatusTimeout);

  // ---- SSE: the last CTA adds the per-tile pairs in tile order (TwoSum)
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
    for (long long i = tid; i < ntiles; i += kThreads) {
      const float2 p = __ldcg(a.part + i);
      two_sum_acc(hi, lo, p.x);
      lo = __fadd_rn(lo, p.y);
    }
    warp_two_sum(hi, lo);
    __shared__ float2 s_fin[kThreads / 32];
    if (lane == 0) s_fin[warp] = make_float2(hi, lo);
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) tot += (double)s_fin[w].x + (double)s_fin[w].y;
      *a.sse = tot;
      *a.ticket = 0u;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)a.ncols);
}

// ------------------------------------------------------------------ host
namespace {

// The driver's tensor-map encoder, looked up once (thread-safe static
// initialisation: server workers call this concurrently).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    cudaDriverEntryPointQueryResult q{};
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
  return fn;
}

template <int NB, int W, int NA>
cudaError_t launch_tcs_t(const CUtensorMap& map, const TcsArgs& a, int grid, size_t smem,
                         cudaStream_t st) {
  cudaError_t e = allow_max_smem(assign_tcs_kernel<NB, W, NA>);
  if (e != cudaSuccess) return e;
  assign_tcs_kernel<NB, W, NA><<<grid, tcs_threads(W), smem, st>>>(map, a);
  return cudaGetLastError();
}

}  // namespace

// Plan of the streaming kernel for (n, k, terms): shared memory (0 if the
// kernel does not take the shape), warpgroups, A buffers, stages and TMEM
// columns.  Rows of at most 32 features get four warpgroups with an A buffer
// each, rows of at most 64 two with one each, wider rows two sharing one.
//
// Stage-ring depth.  A warpgroup converting tile li knows only that tile
// li - NA is converted (its A buffer's previous MMA has completed); the
// tiles in between belong to other warpgroups and may not have landed.  Its
// parity wait on a stage is only sound if the stage's previous use has
// completed, so that use must lie in tile li - NA or earlier, or in its own
// tile: the ring needs at least NA * NB stages when NA > 1 (a shallower ring
// let a wait succeed one phase early).  Every configuration also wants a few
// stages in flight: at least three, two for the last resort.
size_t assign_tcs_plan(int n, int k, int terms, size_t limit, TcsPlan* out) {
  if (n < 1 || n > 128 || n % 4 != 0 || k < 1 || k > 128) return 0;
  const int nb = (n + 31) / 32, N = (k + 15) / 16 * 16;
  const int planes = terms == 3 ? 2 : 1;
  struct Cfg { int w, na, min_stages; };
  Cfg cfgs[3];
  int nc = 0;
  if (nb == 1) cfgs[nc++] = {4, 4, 3};
  if (nb <= 2) cfgs[nc++] = {2, 2, 3};
  cfgs[nc++] = {2, 1, 2};
  for (int i = 0; i < nc; ++i) {
    const Cfg c = cfgs[i];
    if (c.w * N > 512) continue;   // TMEM columns
    const int need = std::max(c.min_stages, c.na > 1 ? c.na * nb : 0);
    if (need > kTcsMaxStages) continue;
    int stages = 0;
    for (int s = kTcsMaxStages; s >= need; --s)
      if ((size_t)tcs_layout(nb, N, k, planes, s, c.na).total + 1024 <= limit) {
        stages = s;
        break;
      }
    if (!stages) continue;
    int ncols = 32;
    while (ncols < c.w * N) ncols <<= 1;
    out->w = c.w;
    out->na = c.na;
    out->stages = stages;
    out->ncols = ncols;
    return (size_t)tcs_layout(nb, N, k, planes, stages, c.na).total + 1024;
  }
  return 0;
}

cudaError_t launch_assign_tcs(const float* X, long long m, int n, const float* C, int cstride,
                              const uint8_t* mask, int k, int32_t* labels, float* dmin,
                              float2* part, double* sse, uint32_t* ticket,
                              unsigned long long* rescored, int* status, int terms,
                              const TcsPlan& plan, size_t smem, int grid, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  // X as a 2-D tensor: dim 0 = features (contiguous), dim 1 = rows; boxes of
  // 32 features x 128 rows, 128-byte swizzle, zeros outside the tensor
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  const cuuint64_t strides[1] = {(cuuint64_t)n * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)kTcsRows};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  TcsArgs a{};
  a.m = m; a.n = n; a.k = k; a.N = (k + 15) / 16 * 16; a.terms = terms;
  a.stages = plan.stages; a.ncols = plan.ncols; a.C = C; a.cstride = cstride; a.mask = mask;
  a.labels = labels; a.dmin = dmin; a.part = part; a.sse = sse; a.ticket = ticket;
  a.rescored = rescored; a.status = status;
  const int nb = (n + 31) / 32;
  if (nb == 1 && plan.w == 4) return launch_tcs_t<1, 4, 4>(map, a, grid, smem, st);
  if (nb == 1 && plan.na == 2) return launch_tcs_t<1, 2, 2>(map, a, grid, smem, st);
  if (nb == 1) return launch_tcs_t<1, 2, 1>(map, a, grid, smem, st);
  if (nb == 2 && plan.na == 2) return launch_tcs_t<2, 2, 2>(map, a, grid, smem, st);
  if (nb == 2) return launch_tcs_t<2, 2, 1>(map, a, grid, smem, st);
  if (nb == 3) return launch_tcs_t<3, 2, 1>(map, a, grid, smem, st);
  return launch_tcs_t<4, 2, 1>(map, a, grid, smem, st);
}

}  // namespace bm
