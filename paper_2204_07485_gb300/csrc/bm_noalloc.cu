// bm_assign_rows_noalloc: the nearest-centroid assignment of bm_assign_rows
// without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need an
// assignment: a process that has handed all of its device memory to its own
// pool allocator up front has none left for the library to take, and a
// latency-critical serving loop cannot afford cudaMalloc / cudaFree, which may
// synchronise the whole device and stall every other stream.  This entry
// point runs the same assignment kernels as bm_assign_rows, but the scratch
// they need -- one float64 partial sum per CTA, the last-CTA ticket and the
// SSE result -- lives in a fixed array compiled into the library.
#include <algorithm>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_internal.h"

namespace bm {

// Scratch capacity: partial sums for up to kNoAllocMaxCtas CTAs, then the
// SSE result (8 bytes) and the ticket (4 bytes).  16,640 bytes per device.
constexpr int kNoAllocMaxCtas = 2048;
constexpr int kNoAllocBytes = 16640;
static_assert(kNoAllocMaxCtas * 8 + 8 + 4 <= kNoAllocBytes, "scratch layout");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current.
constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Every call of the entry point uses the one scratch array, so a call holds
// this lock from its first use of the array (the ticket reset) until its
// result has been read back.  Calls from several host threads -- on one
// stream or on several -- therefore run one after another and never reset
// or read each other's ticket and result.
static std::mutex g_noalloc_call_mu;

static bm_status noalloc_scratch(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BM_ECUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return BM_EUNSUPPORTED;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return BM_ECUDA;
    g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_addr[dev];
  return BM_OK;
}

}  // namespace bm

using namespace bm;

extern "C" bm_status bm_assign_rows_noalloc(const float* X_dev, int64_t m,
                                            int32_t n, const float* C_dev,
                                            const uint8_t* mask_dev, int32_t k,
                                            int32_t* labels_dev,
                                            float* dmin_dev, double* sse_out,
                                            void* stream) {
  if (!X_dev || !C_dev || !mask_dev || m < 1 || n < 1 || k < 1 ||
      m > 2147483647LL)
    return BM_EINVAL;
  if (k > kMaxK) return BM_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> call_lock(g_noalloc_call_mu);
  // at least one live centroid (read into a fixed host buffer)
  uint8_t live_h[kMaxK];
  if (cudaMemcpyAsync(live_h, mask_dev, (size_t)k, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return BM_ECUDA;
  int live = 0;
  for (int j = 0; j < k; ++j) live += live_h[j] != 0;
  if (live == 0) return BM_EINVAL;
  // launch shape: the same kernel family and grid rule as bm_assign_rows
  const bool generic = n > kNpMax;
  const int np = np_width(n);
  const int npad = generic ? align_up(n, 4) : np;
  const int kpad = generic ? align_up(k, 32) : 0;
  const size_t smem = assign_smem(npad, k, kpad, generic);
  if (smem > 227 * 1024) return BM_EUNSUPPORTED;
  const int agrid = assign_max_grid(generic, generic ? 0 : np, smem);
  if (agrid <= 0) return BM_EUNSUPPORTED;
  const long long rows_per = generic ? 64 : 256;
  const int grid = (int)std::max<long long>(1, std::min<long long>(agrid, (m + rows_per - 1) / rows_per));
  if (grid > kNoAllocMaxCtas) return BM_EUNSUPPORTED;   // more CTAs than scratch slots
  unsigned char* base = nullptr;
  bm_status rc = noalloc_scratch(&base);
  if (rc != BM_OK) return rc;
  double* part = reinterpret_cast<double*>(base);
  double* sse = part + kNoAllocMaxCtas;
  uint32_t* ticket = reinterpret_cast<uint32_t*>(sse + 1);
  // the ticket must start at zero; the partials and the result are written
  // before they are read
  if (cudaMemsetAsync(ticket, 0, sizeof(uint32_t), st) != cudaSuccess) return BM_ECUDA;
  AssignArgs a{};
  a.X = X_dev; a.m = m; a.n = n; a.npad = npad; a.k = k; a.kpad = kpad;
  a.C = C_dev; a.cstride = n; a.mask = mask_dev;
  a.labels = labels_dev; a.dmin = dmin_dev;
  a.part = part; a.sse = sse; a.ticket = ticket;
  if (launch_assign(a, grid, generic, generic ? 0 : np, smem, st) != cudaSuccess) return BM_ECUDA;
  double h = 0.0;
  if (cudaMemcpyAsync(&h, sse, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return BM_ECUDA;
  if (sse_out) *sse_out = h;
  return BM_OK;
}
