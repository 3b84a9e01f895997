// The inner PCGP iteration of the mixed mode (Algorithm 3 on the FP32 operators) between two
// F-applies, as one cooperative launch with one CTA per SM.  The phases, each closed by a grid
// barrier (every wait bounded; a wait that gives up sets bit 32 of the error word):
//   body launch only:  P0  Fp = B cbuf (cbuf: the slots of F p), p.Fp, the breakdown test
//                      P1  lambda += gamma p, r -= gamma Fp, the end of the body run (the WHILE
//                          condition of the graph; nothing more once the loop ends)
//   every launch:      P2  gx = G r per subdomain          P3  hx = H gx (dense FP32 H)
//                      P4  w = r - G^T hx and w.w          P4b B^T w at the copy slots (slot-ordered
//                          CSR of B^T)
//                      P5  lumped preconditioner K_bb (B^T w) at the slots, by tasks of up to
//                          kLumpR subdomains that share their boundary blocks (and a row range):
//                          their B^T w placed at their boundary dofs in shared memory, then the
//                          shared blocks applied to all of them at once
//                      P6  z = B cbuf          P7  gx = G z          P8  hx = H gx
//                      P9  y = z - G^T hx, y.w, the stop test     P10  p = y + beta p
// The scalar state (PcgScalar) is read once per launch into shared memory; every CTA runs the
// same scalar logic on the same grid totals (partial sums added in CTA order), and CTA 0 writes
// the state back at the end.  Data written by other CTAs within the launch is read with L2-only
// loads (the L1 caches are not coherent).
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

constexpr int kThreads = 1024;
constexpr unsigned long long kBarSpinLimit = 1ull << 26;

__device__ __noinline__ void grid_sync(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*gen == g0) {
        if (++spins > kBarSpinLimit) {
          atomicOr(err, 32);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Block sum (shuffle tree per warp, then over the warps' sums), returned to every thread.
__device__ __noinline__ double block_sum_all(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Sum of the per-CTA partials part[0 .. gridDim.x) in CTA order, returned to every thread.
__device__ __noinline__ double grid_total(const double* part, double* red) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) s += __ldcg(part + i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  const double t = red[32];
  __syncthreads();
  return t;
}

// (B v)[row] with v read from L2.
__device__ __forceinline__ double b_row_cg(const DevMesh& M, const double* v, long long row) {
  const GroupDev& g = M.groups[M.row_group[row]];
  const int rr = M.row_r[row];
  if (g.dirichlet) return __ldcg(v + g.slot[rr]);
  const int r = rr + 1;
  double s = 0.0;
  for (int j = 0; j <= r; ++j) s += M.helm[r * 8 + j] * __ldcg(v + g.slot[j]);
  return s;
}

// (G^T h)[row] with the padded FP32 values and the padded FP32 h8 (read from L2).
__device__ __forceinline__ double gt_row(const DevMesh& M, const float* h8, long long row) {
  const float4* g4 = reinterpret_cast<const float4*>(M.GTv32);
  const float4* h4 = reinterpret_cast<const float4*>(h8);
  double s = 0.0;
  for (long long e = M.gt_ptr[row]; e < M.gt_ptr[row + 1]; ++e) {
    const int q = __ldg(M.gt_p + e);
    const float4 a = __ldg(g4 + 2 * e), b = __ldg(g4 + 2 * e + 1);
    const float4 u = __ldcg(h4 + 2 * q), v = __ldcg(h4 + 2 * q + 1);
    const float t = a.x * u.x + a.y * u.y + a.z * u.z + a.w * u.w + b.x * v.x + b.y * v.y;
    s += double(t);
  }
  return s;
}

// The row-wise phases, one function for all (the kernel's code stays small enough for the instruction
// caches): kind 0 dst = B cbuf and the sum of other . dst (P0: Fp, p.Fp); 1 dst = src - G^T hx and
// the sum of dst . dst (P4: w); 2 dst = B cbuf (P6: z); 3 dst = src - G^T hx and the sum of
// other . dst (P9: y, y.w).  Two rows per thread and round, their loads issued together.
__device__ __noinline__ double phase_rows(const InnerArgs& a, int kind, const double* src, double* dst,
                                          const double* other, long long gt, long long nthr) {
  const DevMesh& M = a.M;
  const long long m = M.n_mult;
  double acc = 0.0;
#pragma unroll 1
  for (long long r0 = gt; r0 < m; r0 += 2 * nthr) {
    double v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long long row = r0 + u * nthr;
      v[u] = 0.0;
      if (row < m) v[u] = (kind & 1) ? __ldcg(src + row) - gt_row(M, a.hx8, row) : b_row_cg(M, a.cbuf, row);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long long row = r0 + u * nthr;
      if (row >= m) continue;
      dst[row] = v[u];
      if (kind == 1) acc += v[u] * v[u];
      else if (kind != 2) acc += v[u] * __ldcg(other + row);
    }
  }
  return acc;
}

// x += alpha u, y -= alpha v (P1), or p = y + beta p (P10: x = p, u = y, alpha = beta, y null).
__device__ __noinline__ void phase_update(long long m, double alpha, const double* u, double* x, const double* v,
                                          double* y, long long gt, long long nthr) {
#pragma unroll 1
  for (long long row = gt; row < m; row += nthr) {
    if (y) {
      x[row] += alpha * u[row];
      y[row] -= alpha * v[row];
    } else {
      x[row] = u[row] + alpha * x[row];
    }
  }
}

// gx[6p + c] = (G x)[6p + c]: the CTA's subdomains p = blockIdx.x + k grid, kGSub of them at a time,
// the CTA's warps split evenly among them (strided over the subdomain's entries, then warp trees and
// the warps' sums in order).
constexpr int kGSub = 4;
__device__ __noinline__ void phase_G(const InnerArgs& a, const double* x, double* red6) {
  const DevMesh& M = a.M;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int wpg = (int)(blockDim.x >> 5) / kGSub;     // warps per subdomain
  const int gi = w / wpg, wl = w % wpg;               // subdomain slot of this warp, warp within it
  const int nloc = (M.n_sub - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const float4* g4 = reinterpret_cast<const float4*>(M.Gv32);
  for (int k0 = 0; k0 < nloc; k0 += kGSub) {
    const int k = k0 + gi;
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int p = (int)blockIdx.x + k * (int)gridDim.x;
    if (k < nloc) {
      const long long e0 = M.gp_ptr[p], e1 = M.gp_ptr[p + 1];
      float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (long long e = e0 + wl * 32 + l; e < e1; e += 32LL * wpg) {
        const float v = float(__ldcg(x + M.gp_row[e]));
        const float4 ga = __ldg(g4 + 2 * e), gb = __ldg(g4 + 2 * e + 1);
        acc[0] += ga.x * v;
        acc[1] += ga.y * v;
        acc[2] += ga.z * v;
        acc[3] += ga.w * v;
        acc[4] += gb.x * v;
        acc[5] += gb.y * v;
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] = double(acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
      for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
    __syncthreads();
    if (l == 0)
#pragma unroll
      for (int c = 0; c < 6; ++c) red6[c * 32 + w] = s[c];
    __syncthreads();
    if (threadIdx.x < 6 * kGSub) {
      const int sg = threadIdx.x / 6, c = threadIdx.x % 6, kk = k0 + sg;
      if (kk < nloc) {
        double t = 0.0;
        for (int q = 0; q < wpg; ++q) t += red6[c * 32 + sg * wpg + q];
        a.gx[6LL * ((int)blockIdx.x + kk * (int)gridDim.x) + c] = t;
      }
    }
  }
}

// hx = H gx with the FP32 H (rows padded to ld), one warp per row; hx8 the padded FP32 copy.
__device__ __noinline__ void phase_H(const InnerArgs& a, float* xs) {
  for (long long j = threadIdx.x; j < a.ld; j += blockDim.x) xs[j] = j < a.l ? float(__ldcg(a.gx + j)) : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long n4 = a.ld >> 2;
  const float4* x4 = reinterpret_cast<const float4*>(xs);
  for (long long row = (long long)blockIdx.x * nw + (threadIdx.x >> 5); row < a.l; row += (long long)gridDim.x * nw) {
    const float4* a4 = reinterpret_cast<const float4*>(a.H32 + row * a.ld);
    float acc = 0.f;
#pragma unroll 4
    for (long long j = lane; j < n4; j += 32) {
      const float4 h = __ldg(a4 + j), v = x4[j];
      acc += h.x * v.x + h.y * v.y + h.z * v.z + h.w * v.w;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      a.hx[row] = double(acc);
      a.hx8[(row / 6) * 8 + row % 6] = acc;
    }
  }
}

// Lumped preconditioner: cbuf at the copy slots = K_bb (B^T w) for the task's subdomains (boundary
// rows [row0, row1) of the shared blocks, stored [t][c][3 b + a] for stencil neighbour t).
constexpr int kSlotBatch = 4;                     // copy slots per thread per round of loads
// B^T w at every copy slot from the slot-ordered CSR of B^T, kSlotBatch slots per thread at a time:
// their row ranges, first entries and w values each loaded together.
__device__ __noinline__ void phase_slots(const InnerArgs& a, long long gt, long long nthr) {
  const DevMesh& M = a.M;
#pragma unroll 1
  for (long long s0 = gt; s0 < M.n_copy; s0 += nthr * kSlotBatch) {
    int e0[kSlotBatch], e1[kSlotBatch];
#pragma unroll
    for (int u = 0; u < kSlotBatch; ++u) {
      const long long sl = s0 + u * nthr;
      e0[u] = sl < M.n_copy ? __ldg(M.bt_ptr + sl) : 0;
      e1[u] = sl < M.n_copy ? __ldg(M.bt_ptr + sl + 1) : 0;
    }
    int row[kSlotBatch];
    double val[kSlotBatch];
#pragma unroll
    for (int u = 0; u < kSlotBatch; ++u) {
      row[u] = e0[u] < e1[u] ? __ldg(M.bt_row + e0[u]) : 0;
      val[u] = e0[u] < e1[u] ? __ldg(M.bt_val + e0[u]) : 0.0;
    }
    double v[kSlotBatch];
#pragma unroll
    for (int u = 0; u < kSlotBatch; ++u) v[u] = e0[u] < e1[u] ? val[u] * __ldcg(a.w + row[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < kSlotBatch; ++u) {
      for (int e = e0[u] + 1; e < e1[u]; ++e) v[u] += __ldg(M.bt_val + e) * __ldcg(a.w + __ldg(M.bt_row + e));
      const long long sl = s0 + u * nthr;
      if (sl < M.n_copy) a.xslot[sl] = float(v[u]);
    }
  }
}

constexpr int kLumpTG = 4;                        // neighbour groups per row (threads per row)
__device__ __noinline__ void phase_lumped(const InnerArgs& a, float* xs) {
  const DevMesh& M = a.M;
  float* part = xs + (size_t)kLumpR * a.max_nr;     // [kLumpTG][kLumpR][rows per chunk]
  const int ch = blockDim.x / kLumpTG;              // rows per chunk
  const int rl = threadIdx.x % ch, tg = threadIdx.x / ch;
  const int t0 = tg * 7, t1 = min(27, t0 + 7);
  for (int ti = blockIdx.x; ti < a.n_tasks; ti += gridDim.x) {
    const LumpTask* T = a.tasks + ti;
    const int count = T->count, row0 = T->row0, row1 = T->row1;
    long long b2s[kLumpR];
#pragma unroll
    for (int r = 0; r < kLumpR; ++r) b2s[r] = r < count ? M.subs[T->sub[r]].b2s_off : 0;
    const long long bnd_off = M.subs[T->sub[0]].bnd_off;
    const int nr = 3 * M.subs[T->sub[0]].n_bnd;
    __syncthreads();   // the previous task's reads of xs are done
    for (int k = threadIdx.x; k < count * nr; k += blockDim.x) xs[k] = 0.f;   // dofs without a copy slot
    __syncthreads();
    // B^T w at each subdomain's copy slots (contiguous), placed at the slot's boundary dof
#pragma unroll
    for (int r = 0; r < kLumpR; ++r)
      if (r < count) {
        const SubDev& S = M.subs[T->sub[r]];
        for (int q = threadIdx.x; q < S.n_copy; q += blockDim.x) {
          const long long sl = S.copy_off + q;
          xs[r * nr + 3 * __ldg(M.slot_bnd + sl) + q % 3] = __ldcg(a.xslot + sl);
        }
      }
    __syncthreads();
    // rows in chunks of ch, kLumpTG threads per row each taking about a quarter of the 27 stencil
    // neighbours (all their loads issued together), the partial sums added in neighbour order
    const float* kb = a.kbb32 + T->kbb;
    for (int i0 = row0; i0 < row1; i0 += ch) {
      const int i = i0 + rl;
      float acc[kLumpR] = {0.f, 0.f, 0.f, 0.f};
      if (i < row1) {
        const int* tn = M.shape_tnbr + (bnd_off + i / 3) * 27;
#pragma unroll
        for (int t = t0; t < t0 + 7; ++t) {
          if (t >= t1) break;
          const int j = __ldg(tn + t);
          const float k0 = __ldg(kb + (long long)(3 * t) * nr + i), k1 = __ldg(kb + (long long)(3 * t + 1) * nr + i),
                      k2 = __ldg(kb + (long long)(3 * t + 2) * nr + i);
          if (j < 0) continue;
#pragma unroll
          for (int r = 0; r < kLumpR; ++r)
            if (r < count) {
              const float* x = xs + r * nr + 3 * j;
              acc[r] += k0 * x[0] + k1 * x[1] + k2 * x[2];
            }
        }
      }
#pragma unroll
      for (int r = 0; r < kLumpR; ++r) part[(tg * kLumpR + r) * ch + rl] = acc[r];
      __syncthreads();
      if (tg == 0 && i < row1) {
#pragma unroll
        for (int r = 0; r < kLumpR; ++r)
          if (r < count) {
            float v = part[r * ch + rl];
            for (int g = 1; g < kLumpTG; ++g) v += part[(g * kLumpR + r) * ch + rl];
            const int sl = __ldg(M.sub_b2s + b2s[r] + i / 3);
            if (sl >= 0) a.cbuf[(long long)sl + i % 3] = double(v);
          }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_inner(InnerArgs a) {
  extern __shared__ __align__(16) float smem[];
  __shared__ double s_sc[kNumScalars];
  __shared__ double red[33];
  __shared__ double red6[6 * 32];
  __shared__ double s_coef;
  __shared__ int s_more;
  const long long m = a.M.n_mult;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x, nthr = (long long)gridDim.x * blockDim.x;
  const int G = gridDim.x;
  if (threadIdx.x < kNumScalars) s_sc[threadIdx.x] = a.sc[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)a.err & 32) s_sc[kDone] = 1.0;   // an earlier barrier gave up
  __syncthreads();

  if (a.body) {
    // P0: Fp = B cbuf, p.Fp
    {
      const double acc = block_sum_all(phase_rows(a, 0, nullptr, a.Fp, a.p, gt, nthr), red);
      if (threadIdx.x == 0) a.partial[blockIdx.x] = acc;
    }
    grid_sync(a.bar, a.err);
    {
      const double pfp = grid_total(a.partial, red);
      if (threadIdx.x == 0) {
        s_sc[kPFP] = pfp;
        pcg_mid_logic(s_sc);
        s_coef = s_sc[kDone] == 0.0 ? s_sc[kYW] / s_sc[kPFP] : 0.0;
      }
      __syncthreads();
    }
    // P1: the updates (each thread its own rows of P0) and the end of the body run
    if (s_sc[kDone] == 0.0) phase_update(m, s_coef, a.p, a.lam, a.Fp, a.r, gt, nthr);
    __syncthreads();
    if (threadIdx.x == 0) s_more = pcg_post_logic(s_sc) ? 1 : 0;
    __syncthreads();
    const bool more = s_more != 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.has_cond)
      cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, more ? 1u : 0u);
    if (!more) {
      if (blockIdx.x == 0 && threadIdx.x < kNumScalars) a.sc[threadIdx.x] = s_sc[threadIdx.x];
      return;   // every CTA takes this exit (same state)
    }
    grid_sync(a.bar, a.err);
  }
  // P2, P3: hx = H G r
  phase_G(a, a.r, red6);
  grid_sync(a.bar, a.err);
  phase_H(a, smem);
  grid_sync(a.bar, a.err);
  // P4: w = r - G^T hx, w.w
  {
    const double ww = block_sum_all(phase_rows(a, 1, a.r, a.w, nullptr, gt, nthr), red);
    if (threadIdx.x == 0) a.partial[G + blockIdx.x] = ww;
  }
  grid_sync(a.bar, a.err);
  // P4b: B^T w at the copy slots
  phase_slots(a, gt, nthr);
  grid_sync(a.bar, a.err);
  // P5: lumped preconditioner onto the slots
  phase_lumped(a, smem);
  grid_sync(a.bar, a.err);
  // P6: z = B cbuf
  phase_rows(a, 2, nullptr, a.z, nullptr, gt, nthr);
  grid_sync(a.bar, a.err);
  // P7, P8: hx = H G z
  phase_G(a, a.z, red6);
  grid_sync(a.bar, a.err);
  phase_H(a, smem);
  grid_sync(a.bar, a.err);
  // P9: y = z - G^T hx, y.w
  {
    const double yw = block_sum_all(phase_rows(a, 3, a.z, a.y, a.w, gt, nthr), red);
    if (threadIdx.x == 0) a.partial[2 * G + blockIdx.x] = yw;
  }
  grid_sync(a.bar, a.err);
  {
    const double ww = grid_total(a.partial + G, red);
    const double yw = grid_total(a.partial + 2 * G, red);
    if (threadIdx.x == 0) {
      s_sc[kWW] = ww;
      s_sc[kYW] = yw;
      pcg_pre_logic(s_sc);
      s_coef = s_sc[kFirst] != 0.0 ? 0.0 : s_sc[kYW] / s_sc[kYWPrev];
    }
    __syncthreads();
  }
  // P10: p = y + beta p (each thread its own rows of P9)
  if (s_sc[kDone] == 0.0) phase_update(m, s_coef, a.y, a.p, nullptr, nullptr, gt, nthr);
  if (blockIdx.x == 0 && threadIdx.x < kNumScalars) a.sc[threadIdx.x] = s_sc[threadIdx.x];
}

}  // namespace

size_t inner_smem(const InnerArgs& a) {
  const size_t lump = sizeof(float) * ((size_t)kLumpR * (size_t)a.max_nr + (size_t)kLumpR * kThreads);
  const size_t h = sizeof(float) * (size_t)a.ld;
  return std::max(lump, h);
}

int inner_grid(int n_sm, size_t smem) {
  if (cudaFuncSetAttribute(k_inner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_inner, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per >= 1 ? n_sm : 0;
}

cudaError_t launch_inner(const InnerArgs& a, int grid, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_inner, a);
}

}  // namespace tfeti
