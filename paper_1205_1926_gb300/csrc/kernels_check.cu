// Check of the failure detection of bounded device waits: a kernel waits, with the same
// bounded mbarrier wait the F-apply kernels use, on a barrier phase that nothing
// completes; the wait gives up after its limit, the kernel records that and returns.
// No copy is in flight and nothing is left pending, so the context stays usable.
//
// Measurement of the FP64 FMA rate (the roofline of the FP64 kernels): every thread of a
// grid of 4 CTAs per SM runs 16 independent FMA chains; the rate is the flops over the
// CUDA-event time of the launch.
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

// 16 independent chains per thread, x <- x * a + b with |a| < 1 so the values stay bounded; the
// iteration loop is unrolled so that loop control is a small fraction of the issued instructions.
__global__ void k_dfma_rate(int iters, double a, double b, double* out) {
  double x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;   // never true: keeps the chains live
}

}  // namespace

extern "C" int tfeti_measure_fp64_fma(void* cuda_stream, int32_t iters, double* tflops) {
  if (!tflops || iters < 1) return TFETI_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                               cudaSuccess) {
    cudaGetLastError();
    return TFETI_ERR_CUDA;
  }
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return TFETI_ERR_CUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 4 * n_sm, threads = 256;
  k_dfma_rate<<<blocks, threads, 0, st>>>(iters / 10 + 1, 0.999999, 1e-7, d);   // warm-up
  cudaEventRecord(e0, st);
  k_dfma_rate<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, d);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (cudaGetLastError() != cudaSuccess || !(ms > 0.f)) return TFETI_ERR_CUDA;
  *tflops = 2.0 * 16.0 * (double)blocks * threads * (double)iters / (ms * 1e-3) / 1e12;
  return TFETI_OK;
}

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
