// Check of the failure detection of bounded device waits: a kernel waits, with the same
// bounded mbarrier wait the F-apply kernels use, on a barrier phase that nothing
// completes; the wait gives up after its limit, the kernel records that and returns.
// No copy is in flight and nothing is left pending, so the context stays usable.
#include <cuda_runtime.h>

#include "../../include/tfeti.h"
#include "async_common.cuh"

namespace {

__global__ void k_wait_probe(long long limit_cycles, int* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tfeti::mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) out[0] = tfeti::mbar_wait(&bar, 0, limit_cycles) ? 0 : 1;
}

}  // namespace

extern "C" int tfeti_check_bounded_wait(void* cuda_stream, int64_t limit_cycles, int32_t* gave_up) {
  if (!gave_up || limit_cycles < 1 || limit_cycles > (1LL << 31)) return TFETI_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return TFETI_ERR_CUDA;
  }
  cudaMemsetAsync(d, 0xff, sizeof(int), st);
  k_wait_probe<<<1, 32, 0, st>>>(limit_cycles, d);
  int h = -1;
  cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaFree(d);
  if (cudaGetLastError() != cudaSuccess) return TFETI_ERR_CUDA;
  *gave_up = h;
  return TFETI_OK;
}
