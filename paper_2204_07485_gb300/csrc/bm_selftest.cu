// Failure-detection self-test: one grid-barrier wait (the barrier the chunk
// kernels use between phases) whose second participant never arrives.  The
// bounded wait must give up after its time limit, record BM_ETIMEOUT in the
// status word and return, leaving the context usable.  No fault, trap or
// endless loop is involved.
#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_device.cuh"

namespace bm {

__global__ void selftest_wait_kernel(uint32_t* counter, int* status, uint64_t timeout_ns) {
  GridBarrier gb{counter, status, 0u};
  gb.expected = 2;            // a peer CTA that is never launched
  gb.timeout_ns = timeout_ns;
  gb.sync();                  // gives up: status <- kStatusTimeout
}

}  // namespace bm

extern "C" bm_status bm_selftest_wait_timeout(int32_t timeout_ms, void* stream) {
  if (timeout_ms < 1 || timeout_ms > 2000) return BM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* buf = nullptr;
  if (cudaMalloc(&buf, 16) != cudaSuccess) return BM_ENOMEM;
  uint32_t* counter = static_cast<uint32_t*>(buf);
  int* status = reinterpret_cast<int*>(counter + 1);
  bm_status rc = BM_OK;
  if (cudaMemsetAsync(buf, 0, 16, st) != cudaSuccess) rc = BM_ECUDA;
  if (rc == BM_OK) {
    bm::selftest_wait_kernel<<<1, 32, 0, st>>>(counter, status, (uint64_t)timeout_ms * 1000000ull);
    if (cudaGetLastError() != cudaSuccess) rc = BM_ECUDA;
  }
  int h = 0;
  if (rc == BM_OK && (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                      cudaStreamSynchronize(st) != cudaSuccess))
    rc = BM_ECUDA;
  cudaFree(buf);
  if (rc != BM_OK) return rc;
  return h == bm::kStatusTimeout ? BM_ETIMEOUT : (bm_status)h;
}
