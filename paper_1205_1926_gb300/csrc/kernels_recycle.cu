// Start of the dual PCGP from the solver's own history (an extension of
// Algorithm 3, which starts from lambda_Ker = o): the last q solutions
// lambda_j (in Ker N) and their products F lambda_j are kept; for a new
// right-hand side d~ the start lambda0 = sum_j c_j lambda_j minimises the
// F-norm of the error over span{lambda_j}, i.e. (L^T F L) c = L^T d~.  These
// kernels form the small Gram system and the combinations, with fixed-order
// two-stage reductions (bitwise repeatable).
#include "dev.h"

namespace tfeti {

namespace {

constexpr int kRecPairs = kRecMax * kRecMax + kRecMax;   // A (q x q) and b (q)

// partial[block][pair]: pair (i, j) < q*q -> L_i . FL_j ; q*q + i -> L_i . d.
__global__ void __launch_bounds__(256) k_rec_gram_partial(const double* __restrict__ L,
                                                          const double* __restrict__ FL,
                                                          const double* __restrict__ d, int q, long long m,
                                                          double* partial) {
  __shared__ double red[8][kRecPairs];
  double acc[kRecPairs];
#pragma unroll
  for (int p = 0; p < kRecPairs; ++p) acc[p] = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < m; r += (long long)gridDim.x * blockDim.x) {
    double l[kRecMax], fl[kRecMax];
#pragma unroll
    for (int j = 0; j < kRecMax; ++j) {
      l[j] = j < q ? L[(long long)j * m + r] : 0.0;
      fl[j] = j < q ? FL[(long long)j * m + r] : 0.0;
    }
    const double dv = d[r];
#pragma unroll
    for (int i = 0; i < kRecMax; ++i) {
#pragma unroll
      for (int j = 0; j < kRecMax; ++j) acc[i * kRecMax + j] += l[i] * fl[j];
      acc[kRecMax * kRecMax + i] += l[i] * dv;
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < kRecPairs; ++p) {
    double v = acc[p];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][p] = v;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kRecPairs; p += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][p];
    partial[(long long)blockIdx.x * kRecPairs + p] = s;
  }
}

__global__ void k_rec_gram_final(const double* __restrict__ partial, int nblocks, double* out) {
  const int p = threadIdx.x;
  if (p >= kRecPairs) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * kRecPairs + p];
  out[p] = s;
}

// out = (base ? base : 0) + sign * sum_j c_j X_j
__global__ void k_rec_combine(const double* __restrict__ X, const double* __restrict__ c, int q, long long m,
                              const double* __restrict__ base, double sign, double* out) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= m) return;
  double s = 0.0;
  for (int j = 0; j < q; ++j) s += c[j] * X[(long long)j * m + r];
  out[r] = (base ? base[r] : 0.0) + sign * s;
}

}  // namespace

void launch_rec_gram(const double* L, const double* FL, const double* d, int q, long long m, double* partial,
                     double* out, cudaStream_t st) {
  k_rec_gram_partial<<<kRedBlocks, 256, 0, st>>>(L, FL, d, q, m, partial);
  k_rec_gram_final<<<1, 128, 0, st>>>(partial, kRedBlocks, out);
}

void launch_rec_combine(const double* X, const double* c, int q, long long m, const double* base, double sign,
                        double* out, cudaStream_t st) {
  if (m > 0) k_rec_combine<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(X, c, q, m, base, sign, out);
}

}  // namespace tfeti
