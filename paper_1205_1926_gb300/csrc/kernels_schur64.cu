// FP64 F-apply for subdomains that share their shape's elastic factor through the
// shape's dual Schur block S = (K^+)_{boundary,boundary} (formed once in FP64):
// Y = X S with X[k] = B^T lam gathered onto the box-boundary dofs of subdomain k.
// The FLOP count equals that of the two banded sweeps it replaces, but the product
// tiles evenly over all SMs and has no sequential block recurrence, so the FP64
// pipes stay busy.  SIMT DGEMM: 64 x 64 output tile per CTA, K steps of 16,
// 256 threads with 4 x 4 accumulators each, next K step prefetched into registers.
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void k_schur_gather64(DevMesh M, const int* __restrict__ sub_list, int n_list, int n_bd,
                                 const double* __restrict__ lam, double* X) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n_list * n_bd) return;
  const int k = (int)(idx / n_bd), i = (int)(idx % n_bd);
  const SubDev& S = M.subs[sub_list[k]];
  const int sl = M.sub_b2s[S.b2s_off + i / 3];
  X[idx] = sl >= 0 ? bt_at_slot(M, lam, (long long)sl + i % 3) : 0.0;
}

// C = X S (rows: subdomains of sub_list, columns: boundary dofs), scattered to the
// copy slots of the interface dofs.  Sm[j * n_bd + i] = S[i][j] = S[j][i].
__global__ void __launch_bounds__(256) k_schur_dgemm(DevMesh M, const int* __restrict__ sub_list, int n_list,
                                                     int n_bd, const double* __restrict__ X,
                                                     const double* __restrict__ Sm, double* cbuf) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int k0 = blockIdx.y * BM, i0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  double ra[4], rb[4];
  // each thread loads 4 elements of the A tile (64 x 16) and 4 of the B tile (16 x 64)
  auto load = [&](int j0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int am = e / BK, ak = e % BK;
      const int gk = k0 + am, gj = j0 + ak;
      ra[u] = (gk < n_list && gj < n_bd) ? X[(long long)gk * n_bd + gj] : 0.0;
      const int bk = e / BN, bn = e % BN;
      const int gj2 = j0 + bk, gi = i0 + bn;
      rb[u] = (gj2 < n_bd && gi < n_bd) ? Sm[(long long)gj2 * n_bd + gi] : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = threadIdx.x + 256 * u;
      As[buf][e % BK][e / BK] = ra[u];
      Bs[buf][e / BN][e % BN] = rb[u];
    }
  };
  const int nsteps = (n_bd + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int s = 0; s < nsteps; ++s) {
    const int buf = s & 1;
    if (s + 1 < nsteps) load((s + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[buf][kk][ty * 4 + u];
        b[u] = Bs[buf][kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    if (s + 1 < nsteps) store(buf ^ 1);
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
      if (sl >= 0) cbuf[(long long)sl + i % 3] = acc[u][v];
    }
  }
}

}  // namespace

void launch_schur_gather64(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const double* lam, double* X,
                           cudaStream_t st) {
  const long long n = (long long)n_list * n_bd;
  if (n > 0) k_schur_gather64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, sub_list, n_list, n_bd, lam, X);
}

void launch_schur_dgemm_scatter(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const double* X,
                                const double* S, double* cbuf, cudaStream_t st) {
  if (n_list <= 0 || n_bd <= 0) return;
  dim3 grid((unsigned)((n_bd + BN - 1) / BN), (unsigned)((n_list + BM - 1) / BM));
  k_schur_dgemm<<<grid, 256, 0, st>>>(M, sub_list, n_list, n_bd, X, S, cbuf);
}

}  // namespace tfeti
