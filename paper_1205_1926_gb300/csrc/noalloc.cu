// tfeti_apply_projector_noalloc: the coarse projector P_N x = x - G^T H G x
// without any device allocation.
//
// Some callers cannot call cudaMalloc when they apply the operator: a process
// whose device memory is entirely handed to another allocator (a framework's
// caching pool sized to the whole GPU), or a service that forbids allocation
// after start-up so that its memory footprint is fixed.  For them this entry
// point keeps its two coarse-sized work vectors (G x and H G x) in a
// file-scope device array instead of the context's buffers.
//
// The array is static device memory: every GPU that loads the library holds it
// until the process exits, and every call on that GPU shares it.  Calls whose
// kernels overlap on the GPU (different streams without ordering, or two
// contexts used concurrently) race on it.  Both work vectors are fully
// overwritten before they are read, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/tfeti.h"
#include "ctx.h"
#include "dev.h"

namespace {

constexpr long long kMaxCoarse = TFETI_NOALLOC_MAX_COARSE;

// [0, kMaxCoarse): G x;  [kMaxCoarse, 2 kMaxCoarse): H G x.
static __device__ __align__(256) double g_projector_scratch[2 * kMaxCoarse];

// Device address of g_projector_scratch per device, resolved once per device
// with that device current.  Host code must never pass the symbol itself to a
// kernel: on the host it names a stand-in, not device memory.
std::mutex g_mu;
double* g_addr[64] = {nullptr};

int scratch_address(int device, double** out, std::string* why) {
  if (device < 0 || device >= 64) {
    *why = "device ordinal out of range";
    return TFETI_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_projector_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return TFETI_ERR_CUDA;
    }
    g_addr[device] = static_cast<double*>(p);
  }
  *out = g_addr[device];
  return TFETI_OK;
}

int fail_here(tfeti_ctx* c, int code, const std::string& msg) {
  c->err = "tfeti_apply_projector_noalloc: " + msg;
  return code;
}

// Makes the context's device current for the call and puts the caller's device back afterwards.
struct DeviceScope {
  int prev = -1;
  bool switched = false;
  cudaError_t enter(int device) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev == device) return cudaSuccess;
    e = cudaSetDevice(device);
    switched = e == cudaSuccess;
    return e;
  }
  ~DeviceScope() {
    if (switched) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" int tfeti_apply_projector_noalloc(tfeti_ctx* c, const double* x, double* y) {
  if (!c) return TFETI_ERR_ARG;
  if (!x || !y) return fail_here(c, TFETI_ERR_ARG, "null argument");
  if (c->l > kMaxCoarse)
    return fail_here(c, TFETI_ERR_ARG, "coarse size " + std::to_string(c->l) + " exceeds the static limit " +
                                           std::to_string(kMaxCoarse) + " (6 x 4096 subdomains); use "
                                           "tfeti_apply_projector");
  // the scratch address and the launches belong to the context's device, whichever device the
  // caller has current
  DeviceScope scope;
  cudaError_t e = scope.enter(c->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_here(c, TFETI_ERR_CUDA, std::string("selecting the context's device: ") + cudaGetErrorString(e));
  }
  double* scratch = nullptr;
  std::string why;
  const int st = scratch_address(c->device, &scratch, &why);
  if (st != TFETI_OK) return fail_here(c, st, why);
  double* gx = scratch;
  double* hx = scratch + kMaxCoarse;
  tfeti::launch_G_apply(c->M, x, nullptr, gx, 1.0, c->st);
  tfeti::coarse_apply(c->coarse, gx, 1.0, hx, c->st);
  tfeti::launch_GT_update(c->M, x, 1.0, hx, -1.0, y, c->st);
  c->launches += 2 + tfeti::coarse_launches(c->coarse);
  e = cudaGetLastError();                  // launch errors of these three kernels
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_here(c, TFETI_ERR_CUDA, cudaGetErrorString(e));
  }
  return TFETI_OK;
}
