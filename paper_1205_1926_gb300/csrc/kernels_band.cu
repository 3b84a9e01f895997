// Batched banded Cholesky of the regularised subdomain matrices K_rr and the
// generalised-inverse apply K^+ x (Remark 1: fixing dofs replaced by identity
// rows, forward and backward substitution).
//
// Band workspace (per subdomain, n rows, half bandwidth bw, W = bw + 1):
//   band[r*W + k] = K[r][r - bw + k] on input, L[r][r - bw + k] after factorisation.
//
// Factor record written by the factorisation and read by the solves, for row
// blocks b of nb rows (r0 = b nb):
//   panel b : M_b = L_bb^{-1} L_b,off, nb x bw, entry (t, j) = column r0 - bw + j
//   dinv b  : L_bb^{-1}, nb x nb lower triangular
// With L = D (I + N), D = blockdiag(L_bb), N_b = M_b:
//   L^{-1} x = (I + N)^{-1} D^{-1} x   and   L^{-T} y = D^{-T} (I + N)^{-T} y,
// so each step of the forward and backward block recurrences is one GEMV with
// a panel, and the triangular blocks are applied in parallel before and after.
#include <cstdint>

#include "async_common.cuh"
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

constexpr int kThreads = 256;
constexpr int kNB1 = kMaxNB + 1;

// ---------------------------------------------------------------------------
// Factorisation: a cluster of C CTAs per subdomain, right-looking by block
// columns of nb.  Per block column every CTA factors the diagonal block and
// inverts it (identical, deterministic results, no exchange needed); the CTAs
// split the factor-record panel of the block row, the panel TRSM through the
// inverse and the SYRK update of the trailing band.  Two cluster barriers per
// block column order the global-memory band updates between the CTAs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cluster_sync_all() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// Cholesky of the jb x jb block D (lower, in shared memory) and its inverse X, all threads.
// The pivot's square root and reciprocal come from y = 1/sqrt(d) by Newton-Raphson,
// y <- y (3 - d y^2) / 2, two steps from an FP32 rsqrtf guess (2^-23 -> below FP64
// rounding): on this part every FP64 instruction of a lone thread occupies the
// sub-partition's FP64 pipe for a whole warp's worth of cycles, so the library
// square root and division sequences dominated the column step.  A pivot that is
// not positive sets bit 1 of err and is replaced by 1.
__device__ void diag_factor_invert(double* D, double* X, int jb, int* err) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double s_rdiag[kMaxNB];
  // X = I; column c of the factor and row c of X = L^{-1} advance together: after the
  // pivot, column c of L and row c of X are scaled by 1/L[c][c]; then the trailing lower
  // triangle of D and the rows r > c of X (X[r][:] -= L[r][c] X[c][:]) are updated in the
  // same phase, three barriers per column
  for (int e = tid; e < jb * jb; e += nt) X[(e / jb) * kNB1 + e % jb] = (e / jb == e % jb) ? 1.0 : 0.0;
  for (int c = 0; c < jb; ++c) {
    if (tid == 0) {
      double d = D[c * kNB1 + c];
      if (!(d > 0.0)) {
        atomicOr(err, 1);
        d = 1.0;
      }
      double y = (double)rsqrtf((float)d);
      y = y * (1.5 - 0.5 * d * y * y);
      y = y * (1.5 - 0.5 * d * y * y);
      D[c * kNB1 + c] = d * y;
      s_rdiag[c] = y;
    }
    __syncthreads();
    const double inv = s_rdiag[c];
    const int m = jb - c - 1;
    for (int e = tid; e < jb; e += nt) {
      if (e < m) D[(c + 1 + e) * kNB1 + c] *= inv;
      else X[c * kNB1 + (e - m)] *= inv;
    }
    __syncthreads();
    // trailing lower triangle, enumerated densely so that every lane of a warp has an entry,
    // followed by the m x (c + 1) update of X
    const int ntri = m * (m + 1) / 2;
    for (int e = tid; e < ntri + m * (c + 1); e += nt) {
      if (e < ntri) {
        int t = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (t * (t + 1) / 2 > e) --t;
        while ((t + 1) * (t + 2) / 2 <= e) ++t;
        const int r = c + 1 + t, q = c + 1 + (e - t * (t + 1) / 2);
        D[r * kNB1 + q] -= D[r * kNB1 + c] * D[q * kNB1 + c];
      } else {
        const int f = e - ntri, r = c + 1 + f / (c + 1), q = f % (c + 1);
        X[r * kNB1 + q] -= D[r * kNB1 + c] * X[c * kNB1 + q];
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) k_band_chol(DevMesh M, const int* __restrict__ sub_list,
                                                         const long long* __restrict__ off_list, double* band,
                                                         const long long* __restrict__ fac_list, double* fac_pool,
                                                         int* err) {
  extern __shared__ double sm[];
  double* Dm = sm;                       // [NB][NB+1] diagonal block -> its Cholesky factor
  double* Di = Dm + kMaxNB * kNB1;       // [NB][NB+1] inverse of the factor
  double* Lp = Di + kMaxNB * kNB1;       // [bw][NB+1] panel
  const int C = (int)cluster_size(), q = (int)cluster_rank();
  const int item = blockIdx.x / C;
  const int p = sub_list[item];
  const SubDev S = M.subs[p];
  double* A = band + off_list[item];
  double* fac = fac_pool + fac_list[item];
  double* dinv = fac + (long long)S.nblk * S.rec;
  const int n = S.n_dof, bw = S.bw, W = bw + 1, NB = S.nb;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j0 = 0, b = 0; j0 < n; j0 += NB, ++b) {
    const int jb = min(NB, n - j0);
    #pragma unroll 4
    for (int idx = tid; idx < jb * jb; idx += nt) {
      const int r = idx / jb, c = idx % jb;
      Dm[r * kNB1 + c] = (c <= r) ? A[(long long)(j0 + r) * W + c - r + bw] : 0.0;
    }
    __syncthreads();
    diag_factor_invert(Dm, Di, jb, err);
    // factor record of block row b (split over the cluster): dinv and M_b = Di * L[b rows][j0-bw .. j0)
    if (q == 0)
      for (int idx = tid; idx < NB * NB; idx += nt) {
        const int t = idx / NB, u = idx % NB;
        dinv[(long long)b * NB * NB + idx] = (t < jb && u < jb && u <= t) ? Di[t * kNB1 + u] : 0.0;
      }
    double* panel = fac + (long long)b * S.rec;
    {
      const int chunk = (S.rec + C - 1) / C;
      const int lo = q * chunk, hi = min(S.rec, lo + chunk);
      for (int idx = lo + tid; idx < hi; idx += nt) {
        double v = 0.0;
        const int t = idx / bw, j = idx % bw;
        const int c = j0 - bw + j;
        if (idx < NB * bw && t < jb && c >= 0) {
          for (int u = 0; u <= t; ++u) {
            const int k = c - (j0 + u) + bw;
            if (k >= 0) v += Di[t * kNB1 + u] * A[(long long)(j0 + u) * W + k];
          }
        }
        panel[idx] = v;
      }
    }
    const int i0 = j0 + jb;
    const int P = min(bw, n - i0);
    if (P > 0) {
      // panel TRSM, rows split over the cluster: L[i][j0+c] = sum_{s<=c} A[i][j0+s] Di[c][s]
      const int rchunk = (P + C - 1) / C;
      const int t0 = q * rchunk, t1 = min(P, t0 + rchunk);
      #pragma unroll 4
      for (int idx = tid; idx < (t1 - t0) * jb; idx += nt) {
        const int t = t0 + idx / jb, c = idx % jb;
        const int i = i0 + t, k = j0 + c - i + bw;
        Lp[t * kNB1 + c] = (k >= 0) ? A[(long long)i * W + k] : 0.0;
      }
      __syncthreads();
      for (int idx = tid; idx < (t1 - t0) * jb; idx += nt) {
        const int t = t0 + idx / jb, c = idx % jb;
        double v = 0.0;
        for (int s2 = 0; s2 <= c; ++s2) v += Lp[t * kNB1 + s2] * Di[c * kNB1 + s2];
        const int i = i0 + t, k = j0 + c - i + bw;
        if (k >= 0) A[(long long)i * W + k] = v;
      }
    }
    cluster_sync_all();
    if (P > 0) {
      #pragma unroll 4
      for (int idx = tid; idx < P * jb; idx += nt) {
        const int t = idx / jb, c = idx % jb;
        const int i = i0 + t, k = j0 + c - i + bw;
        Lp[t * kNB1 + c] = (k >= 0) ? A[(long long)i * W + k] : 0.0;
      }
      __syncthreads();
      // trailing update A[i][i'] -= sum_c L[i][c] L[i'][c], lower triangle split over the cluster
      const int ntri = P * (P + 1) / 2;
      const int tchunk = (ntri + C - 1) / C;
      const int l0 = q * tchunk, l1 = min(ntri, l0 + tchunk);
      for (int L = l0 + tid; L < l1; L += nt) {
        int t = (int)((sqrtf(8.0f * (float)L + 1.0f) - 1.0f) * 0.5f);
        while (t * (t + 1) / 2 > L) --t;
        while ((t + 1) * (t + 2) / 2 <= L) ++t;
        const int tp = L - t * (t + 1) / 2;
        double v = 0.0;
        for (int c = 0; c < jb; ++c) v += Lp[t * kNB1 + c] * Lp[tp * kNB1 + c];
        const int i = i0 + t, ip = i0 + tp;
        A[(long long)i * W + ip - i + bw] -= v;
      }
    }
    cluster_sync_all();
  }
}

// ---------------------------------------------------------------------------
// Subdomain solve: one CTA applies K^+ to up to kMaxRHS subdomains of one
// shape that share a factor record.  Shared memory: two panel buffers
// (nb x bw doubles each) filled one step ahead by bulk copies, the kMaxRHS
// local vectors, two mbarriers.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_sub_solve(DevMesh M, SolveArgs a) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  __shared__ int s_fail;
  const SolveItem item = a.items[blockIdx.x];
  // unit right-hand sides (in_mode 2, 5) carry dof indices in item.sub[]: the geometry is rep_sub's
  const SubDev& S0 = M.subs[(a.in_mode == 2 || a.in_mode == 5) ? a.rep_sub : item.sub[0]];
  const int n = S0.n_dof, bw = S0.bw, nb = S0.nb, nblk = S0.nblk, rec = S0.rec;
  const int R = item.count;
  const int npad = a.npad;                       // vector stride (largest n of the launch, even)
  T* pan[2] = {sm, sm + a.rec_max};
  T* vec = sm + 2 * a.rec_max;                   // [rcap][npad]
  uint64_t* bar = reinterpret_cast<uint64_t*>(vec + ((a.rcap * npad + 1) & ~1));
  const bool own = (item.fac & kOwnFac) != 0;
  const T* fac = (sizeof(T) == 8 ? reinterpret_cast<const T*>(own ? a.fac_own : a.fac)
                                 : reinterpret_cast<const T*>(own ? a.fac32_own : a.fac32)) +
                 (item.fac & ~kOwnFac);
  const T* dinv = fac + (long long)nblk * rec;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nsteps = 2 * nblk;
  const uint32_t pbytes = (uint32_t)rec * (uint32_t)sizeof(T);

  if (tid == 0) {
    s_fail = 0;
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // step k uses the panel of block k (forward, k < nblk) or 2 nblk - 1 - k (backward)
  auto step_block = [nblk, nsteps](int k) { return k < nblk ? k : nsteps - 1 - k; };
  if (tid == 0) {
    bulk_copy(pan[0], fac, pbytes, &bar[0]);
    bulk_copy(pan[1], fac + (long long)step_block(1) * rec, pbytes, &bar[1]);
  }

  // ---- right-hand sides
  const int n_bd = 3 * S0.n_bnd;
  if (a.in_mode == 2 || a.in_mode == 5) {   // unit vectors at boundary dofs (2) or local dofs (5) item.sub[r]
    for (int r = 0; r < R; ++r)
      for (int i = tid; i < n; i += nt) vec[r * npad + i] = T(0);
    __syncthreads();
    if (tid < R) {
      const int j = item.sub[tid];
      vec[tid * npad + (a.in_mode == 2 ? 3 * M.shape_bln[S0.bnd_off + j / 3] + j % 3 : j)] = T(1);
    }
  }
  const bool unit_in = a.in_mode == 2 || a.in_mode == 5;
  for (int r = 0; r < R && !unit_in; ++r) {
    const SubDev& S = M.subs[item.sub[r]];
    T* x = vec + r * npad;
    if (a.in_mode == 0)
      for (int i = tid; i < n; i += nt) x[i] = T(0);
    else if (a.in_mode == 4)
      for (int i = tid; i < n; i += nt) x[i] = a.bmask[S.dof_off + i] ? T(0) : T(a.src[S.dof_off + i]);
    else
      for (int i = tid; i < n; i += nt) x[i] = a.src ? T(a.src[S.dof_off + i]) : T(0);
  }
  __syncthreads();
  for (int r = 0; r < R && !unit_in; ++r) {
    const SubDev& S = M.subs[item.sub[r]];
    T* x = vec + r * npad;
    if (a.in_mode == 0) {
      for (int s = tid; s < S.n_copy; s += nt) {
        const long long slot = S.copy_off + s;
        x[M.slot_ldof[slot]] = T(bt_at_slot(M, a.lam, slot));
      }
    } else if (a.lam) {
      for (int s = tid; s < S.n_copy; s += nt) {
        const long long slot = S.copy_off + s;
        x[M.slot_ldof[slot]] -= T(bt_at_slot(M, a.lam, slot));
      }
    }
  }
  __syncthreads();
  if (tid < 6 && !a.no_fix)
    for (int r = 0; r < R; ++r) vec[r * npad + S0.fix[tid]] = T(0);
  __syncthreads();

  // ---- x' = D^{-1} x, block-diagonal, 256 rows at a time through registers
  for (int base = 0; base < n; base += nt) {
    const int i = base + tid;
    T v[kMaxRHS] = {T(0), T(0), T(0), T(0)};
    if (i < n) {
      const int b = i / nb, t = i - b * nb, r0 = b * nb;
      const T* drow = dinv + (long long)b * nb * nb + t * nb;
      for (int q = 0; q <= t; ++q) {
        const T d = drow[q];
#pragma unroll
        for (int r = 0; r < kMaxRHS; ++r)
          if (r < R) v[r] = fma(d, vec[r * npad + r0 + q], v[r]);
      }
    }
    __syncthreads();
    if (i < n)
#pragma unroll
      for (int r = 0; r < kMaxRHS; ++r)
        if (r < R) vec[r * npad + i] = v[r];
    __syncthreads();
  }

  // ---- block recurrences: forward y_b = x'_b - M_b y[r0-bw, r0), then backward
  //      z'[r0-bw, r0) -= M_b^T z'_b for b = nblk-1 .. 0
  const int g = lane >> 3, l = lane & 7;
  int k_fail = -1;
  for (int k = 0; k < nsteps; ++k) {
    const int buf = k & 1;
    const bool ok = mbar_wait(&bar[buf], (uint32_t)((k >> 1) & 1));
    if (!ok) s_fail = 1;
    const T* P = pan[buf];
    const int b = step_block(k);
    const int r0 = b * nb, jb = min(nb, n - r0);
    const int c0 = r0 - bw, jlo = max(0, -c0);
    if (ok) {
      if (k < nblk) {
        const int t = 4 * warp + g;                 // 8 warps x 4 rows = 32 rows
        const bool act = t < jb;
        T acc[kMaxRHS] = {T(0), T(0), T(0), T(0)};
        if (act) {
          const T* prow = P + t * bw;
          for (int j = l; j < bw; j += 8) {
            if (j < jlo) continue;
            const T mv = prow[j];
            const int c = c0 + j;
#pragma unroll
            for (int r = 0; r < kMaxRHS; ++r)
              if (r < R) acc[r] = fma(mv, vec[r * npad + c], acc[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < kMaxRHS; ++r) {
          acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], 4);
          acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], 2);
          acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], 1);
        }
        if (act && l == 0)
#pragma unroll
          for (int r = 0; r < kMaxRHS; ++r)
            if (r < R) vec[r * npad + r0 + t] -= acc[r];
      } else {
        // one (column, right-hand side) pair per thread: bw * R units spread evenly over the CTA
        const int units = (bw - jlo) * R;
        for (int u = tid; u < units; u += nt) {
          const int j = jlo + u / R, r = u - (u / R) * R;
          const int c = c0 + j;
          const T* zr = vec + r * npad + r0;
          T acc = T(0);
          for (int t = 0; t < jb; ++t) acc = fma(P[t * bw + j], zr[t], acc);
          vec[r * npad + c] -= acc;
        }
      }
    }
    __syncthreads();
    if (s_fail) {
      k_fail = k;
      break;
    }
    if (tid == 0 && k + 2 < nsteps) bulk_copy(pan[buf], fac + (long long)step_block(k + 2) * rec, pbytes, &bar[buf]);
  }
  if (k_fail >= 0) {
    // a panel copy never completed: report, give the copies still in flight (steps
    // k_fail and k_fail + 1) a bounded time to land, and leave
    if (tid == 0) {
      atomicOr(a.err, 2);
      mbar_wait(&bar[k_fail & 1], (uint32_t)((k_fail >> 1) & 1));
      if (k_fail + 1 < nsteps) mbar_wait(&bar[(k_fail + 1) & 1], (uint32_t)(((k_fail + 1) >> 1) & 1));
    }
    return;
  }

  // ---- z = D^{-T} z'
  for (int base = 0; base < n; base += nt) {
    const int i = base + tid;
    T v[kMaxRHS] = {T(0), T(0), T(0), T(0)};
    if (i < n) {
      const int b = i / nb, t = i - b * nb, r0 = b * nb;
      const int jb = min(nb, n - r0);
      const T* dblk = dinv + (long long)b * nb * nb;
      for (int s = t; s < jb; ++s) {
        const T d = dblk[s * nb + t];
#pragma unroll
        for (int r = 0; r < kMaxRHS; ++r)
          if (r < R) v[r] = fma(d, vec[r * npad + r0 + s], v[r]);
      }
    }
    __syncthreads();
    if (i < n)
#pragma unroll
      for (int r = 0; r < kMaxRHS; ++r)
        if (r < R) vec[r * npad + i] = v[r];
    __syncthreads();
  }
  if (tid < 6 && !a.no_fix)
    for (int r = 0; r < R; ++r) vec[r * npad + S0.fix[tid]] = T(0);
  __syncthreads();

  // ---- outputs
  if (a.out_mode == 4) {   // column item.sub[r] of the dense K^+ of the geometry rep_sub, FP64
    for (int r = 0; r < R; ++r) {
      const long long o = a.s_off + (long long)item.sub[r] * n;
      for (int i = tid; i < n; i += nt) a.S64[o + i] = (double)vec[r * npad + i];
    }
    return;
  }
  if (a.out_mode == 2) {
    for (int r = 0; r < R; ++r) {
      const long long o = a.s_off + (long long)item.sub[r] * n_bd;
      for (int i = tid; i < n_bd; i += nt) {
        const T v = vec[r * npad + 3 * M.shape_bln[S0.bnd_off + i / 3] + i % 3];
        a.S32[o + i] = (float)v;
        if (a.S64) a.S64[o + i] = (double)v;
      }
    }
    return;
  }
  for (int r = 0; r < R; ++r) {
    const int p = item.sub[r];
    const SubDev& S = M.subs[p];
    const T* x = vec + r * npad;
    if (a.out_mode == 0 || a.out_mode == 3) {
      for (int s = tid; s < S.n_copy; s += nt) {
        const long long slot = S.copy_off + s;
        a.cbuf[slot] = double(x[M.slot_ldof[slot]]);
      }
    }
    if (a.out_mode == 1 || a.out_mode == 3) {
      const double* Rb = M.R + S.r_off;
      for (int i = tid; i < n; i += nt) {
        double v = double(x[i]);
        if (a.alpha) {
          const double* al = a.alpha + 6 * (long long)p;
          for (int c = 0; c < 6; ++c) v += Rb[(long long)i * 6 + c] * al[c];
        }
        a.dst[S.dof_off + i] = v;
      }
    }
  }
}

}  // namespace

// The device's opt-in shared-memory limit per block.  Kernels whose dynamic shared memory
// depends on the problem get the largest allowed size as their attribute (not the launch's
// own size), so that launches of different contexts from several host threads cannot
// undercut each other.
int smem_optin_max() {
  static const int v = [] {
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return m;
  }();
  return v;
}

// Largest dynamic shared memory a kernel may be given: the opt-in limit less its static
// shared memory (the two together must not exceed the limit).
int dyn_smem_limit(const void* fn) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return 48 * 1024;
  }
  return smem_optin_max() - (int)fa.sharedSizeBytes;
}

void launch_band_chol(const DevMesh& M, const int* sub_list, int n_list, const long long* band_off_list,
                      double* band, const long long* fac_off_list, double* fac, int* err, int max_bw,
                      int n_sm, cudaStream_t st) {
  if (n_list <= 0) return;
  const size_t smem = sizeof(double) * (2 * kMaxNB * kNB1 + (size_t)max_bw * kNB1);
  static const int lim = dyn_smem_limit((const void*)k_band_chol);
  cudaFuncSetAttribute(k_band_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  const bool big = cudaFuncSetAttribute(k_band_chol, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                   cudaSuccess;
  cudaGetLastError();
  // cluster size: the largest power of two with n_list * C <= 2 * n_sm (at most 16, or 8 if
  // non-portable cluster sizes are unavailable)
  int C = 1;
  const int cmax = big ? 16 : 8;
  while (C < cmax && (long long)n_list * C * 2 <= 2LL * n_sm) C *= 2;
  for (;;) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(n_list * C));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int max_clusters = 0;
    if (C > 1 && (cudaOccupancyMaxActiveClusters(&max_clusters, k_band_chol, &cfg) != cudaSuccess ||
                  max_clusters < 1)) {
      cudaGetLastError();
      C /= 2;
      continue;
    }
    cudaLaunchKernelEx(&cfg, k_band_chol, M, sub_list, band_off_list, band, fac_off_list, fac, err);
    return;
  }
}

size_t sub_solve_smem(int rec_max, int npad, int rcap, int elem_bytes) {
  const size_t vec = ((size_t)rcap * npad + 1) & ~(size_t)1;
  return (size_t)elem_bytes * (2 * (size_t)rec_max + vec) + 2 * sizeof(uint64_t);
}

void launch_sub_solve(const DevMesh& M, const SolveArgs& a, size_t smem_bytes, cudaStream_t st) {
  if (a.n_items <= 0) return;
  if (a.fp32) {
    static const int lim = dyn_smem_limit((const void*)k_sub_solve<float>);
    cudaFuncSetAttribute(k_sub_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    k_sub_solve<float><<<a.n_items, kThreads, smem_bytes, st>>>(M, a);
  } else {
    static const int lim = dyn_smem_limit((const void*)k_sub_solve<double>);
    cudaFuncSetAttribute(k_sub_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    k_sub_solve<double><<<a.n_items, kThreads, smem_bytes, st>>>(M, a);
  }
}

namespace {
__global__ void k_to_f32(const double* __restrict__ src, float* dst, const long long* __restrict__ off,
                         long long len) {
  const long long base = off[blockIdx.y];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[base + i] = (float)src[base + i];
}
}  // namespace

void launch_fac_to_f32(const double* fac, float* fac32, const long long* off_list, int n_list, long long len,
                       cudaStream_t st) {
  if (n_list <= 0) return;
  dim3 grid(64, n_list);
  k_to_f32<<<grid, 256, 0, st>>>(fac, fac32, off_list, len);
}

namespace {
__global__ void k_to_f32_flat(const double* __restrict__ src, float* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
}  // namespace

void launch_to_f32(const double* src, float* dst, long long n, cudaStream_t st) {
  if (n > 0) k_to_f32_flat<<<1024, 256, 0, st>>>(src, dst, n);
}

}  // namespace tfeti
