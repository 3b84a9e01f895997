// Batched banded Cholesky of the regularised subdomain matrices K_rr and the
// generalised-inverse apply K^+ x (Remark 1: fixing dofs replaced by identity
// rows, forward and backward substitution).
//
// Band layout (per subdomain, n rows, half bandwidth bw, W = bw + 1):
//   band[r*W + k] = L[r][r - bw + k], k = 0..bw.
// After factorisation the lower triangle of every NB x NB diagonal block
// [j0, j0+NB) holds the inverse of that block of L instead of L itself, so
// that both substitutions become block-row GEMVs with no sequential
// triangle inside a block.
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

constexpr int kThreads = 256;
constexpr int kNB1 = kMaxNB + 1;

// One CTA factorises one subdomain band in place (right-looking, block
// column of NB at a time: diagonal block Cholesky + its inverse, panel TRSM
// through that inverse, SYRK update of the trailing band).
__global__ void __launch_bounds__(kThreads) k_band_chol(DevMesh M, const int* __restrict__ sub_list,
                                                         const long long* __restrict__ off_list, double* band,
                                                         int* err) {
  extern __shared__ double sm[];
  double* Dm = sm;                       // [NB][NB+1] diagonal block -> its Cholesky factor
  double* Di = Dm + kMaxNB * kNB1;       // [NB][NB+1] inverse of the factor
  double* Lp = Di + kMaxNB * kNB1;       // [bw][NB+1] panel
  const int p = sub_list[blockIdx.x];
  const SubDev S = M.subs[p];
  double* A = band + off_list[blockIdx.x];
  const int n = S.n_dof, bw = S.bw, W = bw + 1, NB = S.nb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = min(NB, n - j0);
    for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
      const int r = idx / jb, c = idx % jb;
      Dm[r * kNB1 + c] = (c <= r) ? A[(long long)(j0 + r) * W + c - r + bw] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      for (int c = 0; c < jb; ++c) {
        double d = Dm[c * kNB1 + c];
        if (!(d > 0.0)) {
          if (lane == 0) atomicOr(err, 1);
          d = 1.0;
        }
        d = sqrt(d);
        const double inv = 1.0 / d;
        __syncwarp();
        if (lane == c) Dm[c * kNB1 + c] = d;
        if (lane > c && lane < jb) Dm[lane * kNB1 + c] *= inv;
        __syncwarp();
        if (lane > c && lane < jb) {
          const double lrc = Dm[lane * kNB1 + c];
          for (int s = c + 1; s <= lane; ++s) Dm[lane * kNB1 + s] -= lrc * Dm[s * kNB1 + c];
        }
        __syncwarp();
      }
      // inverse of the lower-triangular factor, one column per lane
      if (lane < jb) {
        const int s = lane;
        for (int r = 0; r < jb; ++r) {
          if (r < s) {
            Di[r * kNB1 + s] = 0.0;
          } else {
            double acc = (r == s) ? 1.0 : 0.0;
            for (int t = s; t < r; ++t) acc -= Dm[r * kNB1 + t] * Di[t * kNB1 + s];
            Di[r * kNB1 + s] = acc / Dm[r * kNB1 + r];
          }
        }
      }
    }
    __syncthreads();
    for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
      const int r = idx / jb, c = idx % jb;
      if (c <= r) A[(long long)(j0 + r) * W + c - r + bw] = Di[r * kNB1 + c];
    }
    const int i0 = j0 + jb;
    const int P = min(bw, n - i0);
    if (P <= 0) {
      __syncthreads();
      continue;
    }
    for (int idx = tid; idx < P * jb; idx += blockDim.x) {
      const int t = idx / jb, c = idx % jb;
      const int i = i0 + t, k = j0 + c - i + bw;
      Lp[t * kNB1 + c] = (k >= 0) ? A[(long long)i * W + k] : 0.0;
    }
    __syncthreads();
    // panel: L[i][j0+c] = sum_{s<=c} A[i][j0+s] Di[c][s]
    for (int t = warp; t < P; t += nwarps) {
      double val = 0.0;
      if (lane < jb)
        for (int s = 0; s <= lane; ++s) val += Lp[t * kNB1 + s] * Di[lane * kNB1 + s];
      __syncwarp();
      if (lane < jb) Lp[t * kNB1 + lane] = val;
    }
    __syncthreads();
    for (int idx = tid; idx < P * jb; idx += blockDim.x) {
      const int t = idx / jb, c = idx % jb;
      const int i = i0 + t, k = j0 + c - i + bw;
      if (k >= 0) A[(long long)i * W + k] = Lp[t * kNB1 + c];
    }
    // trailing update A[i][i'] -= sum_c L[i][c] L[i'][c] over the panel rows (i >= i')
    const int ntri = P * (P + 1) / 2;
    for (int L = tid; L < ntri; L += blockDim.x) {
      int t = (int)((sqrtf(8.0f * (float)L + 1.0f) - 1.0f) * 0.5f);
      while (t * (t + 1) / 2 > L) --t;
      while ((t + 1) * (t + 2) / 2 <= L) ++t;
      const int tp = L - t * (t + 1) / 2;
      double s = 0.0;
      for (int c = 0; c < jb; ++c) s += Lp[t * kNB1 + c] * Lp[tp * kNB1 + c];
      const int i = i0 + t, ip = i0 + tp;
      A[(long long)i * W + ip - i + bw] -= s;
    }
    __syncthreads();
  }
}

// One CTA applies K_p^+ of one subdomain.
__global__ void __launch_bounds__(kThreads) k_sub_solve(DevMesh M, SolveArgs a) {
  extern __shared__ double x[];
  const int p = blockIdx.x;
  const SubDev S = M.subs[p];
  const int n = S.n_dof, bw = S.bw, W = bw + 1, NB = S.nb;
  double* acc = x + ((n + 1) & ~1);
  const double* L = a.band + a.kdag_off[p];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (a.in_mode == 0) {
    for (int i = tid; i < n; i += blockDim.x) x[i] = 0.0;
    __syncthreads();
    for (int s = tid; s < S.n_copy; s += blockDim.x) {
      const long long slot = S.copy_off + s;
      x[M.slot_ldof[slot]] = bt_at_slot(M, a.lam, slot);
    }
  } else {
    for (int i = tid; i < n; i += blockDim.x) x[i] = a.src ? a.src[S.dof_off + i] : 0.0;
    __syncthreads();
    if (a.lam)
      for (int s = tid; s < S.n_copy; s += blockDim.x) {
        const long long slot = S.copy_off + s;
        x[M.slot_ldof[slot]] -= bt_at_slot(M, a.lam, slot);
      }
  }
  __syncthreads();
  if (tid < 6) x[S.fix[tid]] = 0.0;
  __syncthreads();
  // forward: L y = x, block rows of NB
  for (int r0 = 0; r0 < n; r0 += NB) {
    const int jb = min(NB, n - r0);
    for (int t = warp; t < jb; t += nwarps) {
      const int i = r0 + t;
      const double* row = L + (long long)i * W - i + bw;   // row[c] = L[i][c]
      double s = 0.0;
      for (int c = max(0, i - bw) + lane; c < r0; c += 32) s += row[c] * x[c];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) acc[t] = x[i] - s;
    }
    __syncthreads();
    if (tid < jb) {
      const int i = r0 + tid;
      const double* row = L + (long long)i * W - i + bw;
      double s = 0.0;
      for (int q = 0; q <= tid; ++q) s += row[r0 + q] * acc[q];
      x[i] = s;
    }
    __syncthreads();
  }
  // backward: L^T z = y, block rows from the bottom
  for (int r0 = ((n - 1) / NB) * NB; r0 >= 0; r0 -= NB) {
    const int jb = min(NB, n - r0);
    if (tid < jb) {
      const int c = tid;
      double s = 0.0;
      for (int t = c; t < jb; ++t) s += L[(long long)(r0 + t) * W + c - t + bw] * x[r0 + t];
      acc[c] = s;
    }
    __syncthreads();
    if (tid < jb) x[r0 + tid] = acc[tid];
    __syncthreads();
    for (int c = max(0, r0 - bw) + tid; c < r0; c += blockDim.x) {
      double s = 0.0;
      for (int t = 0; t < jb; ++t) {
        const int i = r0 + t;
        if (c >= i - bw) s += L[(long long)i * W + c - i + bw] * x[i];
      }
      x[c] -= s;
    }
    __syncthreads();
  }
  if (tid < 6) x[S.fix[tid]] = 0.0;
  __syncthreads();
  if (a.out_mode == 0) {
    for (int s = tid; s < S.n_copy; s += blockDim.x) {
      const long long slot = S.copy_off + s;
      a.cbuf[slot] = x[M.slot_ldof[slot]];
    }
  } else {
    const double* R = M.R + S.r_off;
    for (int i = tid; i < n; i += blockDim.x) {
      double v = x[i];
      if (a.alpha) {
        const double* al = a.alpha + 6 * (long long)p;
        for (int c = 0; c < 6; ++c) v += R[(long long)i * 6 + c] * al[c];
      }
      a.dst[S.dof_off + i] = v;
    }
  }
}

}  // namespace

void launch_band_chol(const DevMesh& M, const int* sub_list, int n_list, const long long* band_off_list,
                      double* band, int* err, int max_bw, cudaStream_t st) {
  if (n_list <= 0) return;
  const size_t smem = sizeof(double) * (2 * kMaxNB * kNB1 + (size_t)max_bw * kNB1);
  cudaFuncSetAttribute(k_band_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_band_chol<<<n_list, kThreads, smem, st>>>(M, sub_list, band_off_list, band, err);
}

void launch_sub_solve(const DevMesh& M, const SolveArgs& a, int max_ndof, cudaStream_t st) {
  const size_t smem = sizeof(double) * ((size_t)((max_ndof + 1) & ~1) + kMaxNB);
  cudaFuncSetAttribute(k_sub_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_sub_solve<<<M.n_sub, kThreads, smem, st>>>(M, a);
}

}  // namespace tfeti
