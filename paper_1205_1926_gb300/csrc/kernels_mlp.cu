// Per-interface MLP of the learned start: for every multiplier row a small network
// maps local features (previous-step interface increments, the dual right-hand
// side, the load-increment ratio, local plastic indicators) to a predicted entry
// of lambda_Ker for the first Newton solve of the next load step.  The
// prediction only enters the Galerkin start of the dual PCGP as one more basis
// vector, so the start is still compared against the zero start of Algorithm 3.
//
// Network: kMlpIn -> kMlpHid (ReLU) -> kMlpHid (ReLU) -> 1, in residual form: the
// output is f0 (the previous step's value) plus the network, whose last layer starts
// at zero, so the untrained predictor is "as in the previous load step".  Inference reads FP16
// copies of the weights and accumulates in FP32; training keeps FP32 master
// weights with Adam.  Gradients are summed in a fixed order (per-CTA partial sums,
// then one ordered reduction), so training is bitwise repeatable.
#include <cuda_fp16.h>

#include "dev.h"

namespace tfeti {

namespace {

constexpr int kIn = kMlpIn, kHid = kMlpHid;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid;
static_assert(kOffB3 + 1 == kMlpParams, "parameter layout");

// Features of row r: f0 = la/s, f1 = (la - lb)/s, f2 = d/sd, f3 = rho, f4 = plastic
// fraction now, f5 = plastic fraction at the previous step (max over the
// subdomains of the row's group), f6 = Newton-index feature, zero padding.
__device__ __forceinline__ void row_features(const DevMesh& M, long long r, const double* la, const double* lb,
                                             const double* d, const float* pf_now, const float* pf_prev,
                                             const float* scal, float* x) {
  const GroupDev& g = M.groups[M.row_group[r]];
  float pn = 0.f, pp = 0.f;
  for (int j = 0; j < g.k; ++j) {
    pn = fmaxf(pn, pf_now[g.sub[j]]);
    pp = fmaxf(pp, pf_prev[g.sub[j]]);
  }
  const float inv_s = scal[0], inv_sd = scal[1];
  x[0] = (float)la[r] * inv_s;
  x[1] = (float)(la[r] - lb[r]) * inv_s;
  x[2] = (float)d[r] * inv_sd;
  x[3] = scal[2];
  x[4] = pn;
  x[5] = pp;
  x[6] = scal[4];
#pragma unroll
  for (int k = 7; k < kIn; ++k) x[k] = 0.f;
}

// y[r] = s * net(x_r): one thread per row, FP16 weights staged in shared memory.
__global__ void __launch_bounds__(256) k_mlp_infer(DevMesh M, const __half* __restrict__ w16, const double* la,
                                                   const double* lb, const double* d, const float* pf_now,
                                                   const float* pf_prev, const float* scal, double* y) {
  __shared__ float w[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = __half2float(w16[i]);
  __syncthreads();
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= M.n_mult) return;
  float x[kIn], h1[kHid];
  row_features(M, r, la, lb, d, pf_now, pf_prev, scal, x);
#pragma unroll 4
  for (int j = 0; j < kHid; ++j) {
    float a = w[kOffB1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(w[kOffW1 + j * kIn + k], x[k], a);
    h1[j] = fmaxf(a, 0.f);
  }
  float out = x[0] + w[kOffB3];    // residual form: the previous step's value plus the network's correction
  for (int j = 0; j < kHid; ++j) {
    float a = w[kOffB2 + j];
#pragma unroll
    for (int k = 0; k < kHid; ++k) a = fmaf(w[kOffW2 + j * kHid + k], h1[k], a);
    out = fmaf(w[kOffW3 + j], fmaxf(a, 0.f), out);
  }
  y[r] = (double)out * (double)scal[3];
}

// One minibatch of kMlpBatch rows per CTA (rows drawn with a fixed stride from
// `start`), forward + backward of the mean squared error against t_r / s; the
// CTA's gradient goes to partial[blockIdx.x][kMlpParams].
__global__ void __launch_bounds__(kMlpBatch) k_mlp_grad(DevMesh M, const float* __restrict__ wm, const double* la,
                                                        const double* lb, const double* d, const float* pf_now,
                                                        const float* pf_prev, const float* scal, const double* target,
                                                        long long start, long long stride, float* partial) {
  extern __shared__ float sm[];
  float* w = sm;                                   // [kMlpParams]
  float* X = w + kMlpParams;                       // [kMlpBatch][kIn]
  float* H1 = X + kMlpBatch * kIn;                 // [kMlpBatch][kHid]  post-ReLU
  float* D2 = H1 + kMlpBatch * kHid;               // [kMlpBatch][kHid]  dL/d(pre-activation 2)
  float* D1 = D2 + kMlpBatch * kHid;               // [kMlpBatch][kHid]  dL/d(pre-activation 1)
  float* DY = D1 + kMlpBatch * kHid;               // [kMlpBatch]
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = wm[i];
  __syncthreads();
  const int b = threadIdx.x;
  const long long r = (start + ((long long)blockIdx.x * kMlpBatch + b) * stride) % M.n_mult;
  float x[kIn];
  row_features(M, r, la, lb, d, pf_now, pf_prev, scal, x);
  for (int k = 0; k < kIn; ++k) X[b * kIn + k] = x[k];
  float h1[kHid], h2[kHid];
  for (int j = 0; j < kHid; ++j) {
    float a = w[kOffB1 + j];
    for (int k = 0; k < kIn; ++k) a = fmaf(w[kOffW1 + j * kIn + k], x[k], a);
    h1[j] = fmaxf(a, 0.f);
    H1[b * kHid + j] = h1[j];
  }
  float out = x[0] + w[kOffB3];
  for (int j = 0; j < kHid; ++j) {
    float a = w[kOffB2 + j];
    for (int k = 0; k < kHid; ++k) a = fmaf(w[kOffW2 + j * kHid + k], h1[k], a);
    h2[j] = a;
    out = fmaf(w[kOffW3 + j], fmaxf(a, 0.f), out);
  }
  const float dy = (out - (float)target[r] * scal[0]) * (2.0f / (float)(gridDim.x * kMlpBatch));
  DY[b] = dy;
  for (int j = 0; j < kHid; ++j) D2[b * kHid + j] = h2[j] > 0.f ? dy * w[kOffW3 + j] : 0.f;
  // keep h2 (post-ReLU) for dW3 in the D1 rows until dh1 overwrites them
  for (int j = 0; j < kHid; ++j) D1[b * kHid + j] = fmaxf(h2[j], 0.f);
  __syncthreads();
  float* g = partial + (long long)blockIdx.x * kMlpParams;
  // dW3, db3
  for (int j = threadIdx.x; j < kHid; j += blockDim.x) {
    float s = 0.f;
    for (int bb = 0; bb < kMlpBatch; ++bb) s += DY[bb] * D1[bb * kHid + j];
    g[kOffW3 + j] = s;
  }
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int bb = 0; bb < kMlpBatch; ++bb) s += DY[bb];
    g[kOffB3] = s;
  }
  // dW2[j][k] = sum_b D2[b][j] H1[b][k], db2
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int j = e / kHid, k = e % kHid;
    float s = 0.f;
    for (int bb = 0; bb < kMlpBatch; ++bb) s += D2[bb * kHid + j] * H1[bb * kHid + k];
    g[kOffW2 + e] = s;
  }
  for (int j = threadIdx.x; j < kHid; j += blockDim.x) {
    float s = 0.f;
    for (int bb = 0; bb < kMlpBatch; ++bb) s += D2[bb * kHid + j];
    g[kOffB2 + j] = s;
  }
  __syncthreads();
  // dh1 = W2^T D2, masked by ReLU'
  for (int k = 0; k < kHid; ++k) {
    float s = 0.f;
    for (int j = 0; j < kHid; ++j) s = fmaf(w[kOffW2 + j * kHid + k], D2[b * kHid + j], s);
    D1[b * kHid + k] = H1[b * kHid + k] > 0.f ? s : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x) {
    const int j = e / kIn, k = e % kIn;
    float s = 0.f;
    for (int bb = 0; bb < kMlpBatch; ++bb) s += D1[bb * kHid + j] * X[bb * kIn + k];
    g[kOffW1 + e] = s;
  }
  for (int j = threadIdx.x; j < kHid; j += blockDim.x) {
    float s = 0.f;
    for (int bb = 0; bb < kMlpBatch; ++bb) s += D1[bb * kHid + j];
    g[kOffB1 + j] = s;
  }
}

// Sum the CTA gradients in order and take one Adam step (step count t >= 1);
// refresh the FP16 copy.
__global__ void k_mlp_adam(const float* __restrict__ partial, int nparts, float* wm, float* m1, float* m2,
                           __half* w16, float lr, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  float gsum = 0.f;
  for (int p = 0; p < nparts; ++p) gsum += partial[(long long)p * kMlpParams + i];
  const float b1 = 0.9f, b2 = 0.999f;
  const float a = b1 * m1[i] + (1.f - b1) * gsum;
  const float v = b2 * m2[i] + (1.f - b2) * gsum * gsum;
  m1[i] = a;
  m2[i] = v;
  const float ah = a / (1.f - powf(b1, (float)t)), vh = v / (1.f - powf(b2, (float)t));
  const float wn = wm[i] - lr * ah / (sqrtf(vh) + 1e-8f);
  wm[i] = wn;
  w16[i] = __float2half(wn);
}

// Per-subdomain plastic fraction from the per-subdomain plastic Gauss-point counts.
__global__ void k_plastic_fraction(DevMesh M, const int* __restrict__ sub_np, float* pf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M.n_sub) return;
  pf[p] = (float)sub_np[p] / (float)(8 * M.subs[p].n_elem);
}

__global__ void k_mlp_cast(const float* __restrict__ wm, __half* w16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kMlpParams) w16[i] = __float2half(wm[i]);
}

}  // namespace

size_t mlp_grad_smem() {
  return sizeof(float) * (kMlpParams + kMlpBatch * kIn + 3 * kMlpBatch * kHid + kMlpBatch);
}

void launch_mlp_infer(const DevMesh& M, const void* w16, const double* la, const double* lb, const double* d,
                      const float* pf_now, const float* pf_prev, const float* scal, double* y, cudaStream_t st) {
  if (M.n_mult > 0)
    k_mlp_infer<<<(unsigned)((M.n_mult + 255) / 256), 256, 0, st>>>(M, static_cast<const __half*>(w16), la, lb, d,
                                                                      pf_now, pf_prev, scal, y);
}

void launch_mlp_train_step(const DevMesh& M, const float* wm, const double* la, const double* lb, const double* d,
                           const float* pf_now, const float* pf_prev, const float* scal, const double* target,
                           long long start, long long stride, int nblocks, float* partial, float* wm_out, float* m1,
                           float* m2, void* w16, float lr, int t, cudaStream_t st) {
  if (M.n_mult <= 0 || nblocks <= 0) return;
  const size_t smem = mlp_grad_smem();
  cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_mlp_grad<<<nblocks, kMlpBatch, smem, st>>>(M, wm, la, lb, d, pf_now, pf_prev, scal, target, start, stride,
                                               partial);
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(partial, nblocks, wm_out, m1, m2, static_cast<__half*>(w16),
                                                        lr, t);
}

void launch_plastic_fraction(const DevMesh& M, const int* sub_np, float* pf, cudaStream_t st) {
  if (M.n_sub > 0) k_plastic_fraction<<<(M.n_sub + 255) / 256, 256, 0, st>>>(M, sub_np, pf);
}

void launch_mlp_cast(const float* wm, void* w16, cudaStream_t st) {
  k_mlp_cast<<<(kMlpParams + 255) / 256, 256, 0, st>>>(wm, static_cast<__half*>(w16));
}

}  // namespace tfeti
