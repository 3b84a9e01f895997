// Inner F-apply of the mixed-precision PCGP for subdomains that share their
// shape's elastic factor: with S = (K^+)_{boundary,boundary} of the shape (formed
// once in FP64, stored FP32), the subdomain part of F = B K^+ B^T for all such
// subdomains is one FP32 GEMM  Y = X S,  X[k] = B^T lam gathered onto the box
// boundary dofs of subdomain k (zero off its interface).  S is symmetric.
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

__global__ void k_schur_gather(DevMesh M, const int* __restrict__ sub_list, int n_list, int n_bd,
                               const double* __restrict__ lam, float* X) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n_list * n_bd) return;
  const int k = (int)(idx / n_bd), i = (int)(idx % n_bd);
  const SubDev& S = M.subs[sub_list[k]];
  const int sl = M.sub_b2s[S.b2s_off + i / 3];
  X[idx] = sl >= 0 ? (float)bt_at_slot(M, lam, (long long)sl + i % 3) : 0.0f;
}

constexpr int BM = 64, BN = 64, BK = 16;

// C = X S (rows k: subdomains, columns i: boundary dofs), written to the copy
// slots of the interface dofs.  256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) k_schur_gemm(DevMesh M, const int* __restrict__ sub_list, int n_list,
                                                    int n_bd, const float* __restrict__ X,
                                                    const float* __restrict__ Sm, double* cbuf) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int k0 = blockIdx.y * BM, i0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int j0 = 0; j0 < n_bd; j0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int m = e / BK, kk = e % BK;
      const int gk = k0 + m, gj = j0 + kk;
      As[kk][m] = (gk < n_list && gj < n_bd) ? X[(long long)gk * n_bd + gj] : 0.0f;
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      const int kk = e / BN, nn = e % BN;
      const int gj = j0 + kk, gi = i0 + nn;
      Bs[kk][nn] = (gj < n_bd && gi < n_bd) ? Sm[(long long)gj * n_bd + gi] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int k = k0 + ty * 4 + u;
    if (k >= n_list) continue;
    const SubDev& S = M.subs[sub_list[k]];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + tx * 4 + v;
      if (i >= n_bd) continue;
      const int sl = M.sub_b2s[S.b2s_off + i / 3];
      if (sl >= 0) cbuf[(long long)sl + i % 3] = (double)acc[u][v];
    }
  }
}

}  // namespace

void launch_schur_gather(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const double* lam, float* X,
                         cudaStream_t st) {
  const long long n = (long long)n_list * n_bd;
  if (n > 0) k_schur_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, sub_list, n_list, n_bd, lam, X);
}

void launch_schur_gemm_scatter(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const float* X,
                               const float* S, double* cbuf, cudaStream_t st) {
  if (n_list <= 0) return;
  dim3 grid((unsigned)((n_bd + BN - 1) / BN), (unsigned)((n_list + BM - 1) / BM));
  k_schur_gemm<<<grid, 256, 0, st>>>(M, sub_list, n_list, n_bd, X, S, cbuf);
}

}  // namespace tfeti
