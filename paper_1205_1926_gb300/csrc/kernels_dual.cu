// Dual-space kernels of Algorithm 3: B (copy slots -> multipliers), the
// coarse operators G = R^T B^T and G^T, the projector pieces, the lumped
// preconditioner B K B^T, deterministic reductions and the PCGP updates, and
// the one-time coarse set-up (G G^T assembly, dense Cholesky, explicit inverse).
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// y[row] = (B v)[row]
__global__ void k_contract(DevMesh M, const double* __restrict__ v, double* y) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row < M.n_mult) y[row] = b_at_row(M, v, row);
}

__device__ double block_reduce_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;   // valid in thread 0
}

// Six block sums at once, in the order of block_reduce_sum (shuffle tree within each
// warp, then a shuffle tree over the warps' partials), with one barrier; red holds
// 6 x 32 doubles.  The sums are valid in thread 0.
__device__ void block_reduce_sum6(double v[6], double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  if (l == 0)
#pragma unroll
    for (int c = 0; c < 6; ++c) red[c * 32 + w] = v[c];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double s = threadIdx.x < nw ? red[c * 32 + threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[c] = s;
    }
  }
}

// block_reduce_sum6 in FP32: red holds 6 x 32 floats.
__device__ void block_reduce_sum6f(float v[6], float* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  if (l == 0)
#pragma unroll
    for (int c = 0; c < 6; ++c) red[c * 32 + w] = v[c];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float s = threadIdx.x < nw ? red[c * 32 + threadIdx.x] : 0.f;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[c] = s;
    }
  }
}

// gx[6p+c] = scale * (R_p^T x_p)_c over all dofs of subdomain p (set-up: e = -R^T f).
// One CTA per subdomain.
__global__ void k_G_full(DevMesh M, const double* __restrict__ x_full, double* gx, double scale) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  const SubDev S = M.subs[p];
  const double* R = M.R + S.r_off;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < S.n_dof; i += blockDim.x) {
    const double v = x_full[S.dof_off + i];
    const double* r = R + (long long)i * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += r[c] * v;
  }
  for (int c = 0; c < 6; ++c) {
    const double s = block_reduce_sum(acc[c], red);
    if (threadIdx.x == 0) gx[6 * (long long)p + c] = scale * s;
  }
}

// gx[6p+c] = scale * (G x)[6p+c] = scale * sum over the entries of subdomain p of G[entry][c] x[row]
// (and, with gx32, its FP32 rounding for the FP32 coarse GEMV).  One CTA per subdomain.  T: FP64
// values, or their FP32 copy (products, per-thread and block sums in T) for the inner iterations of
// the mixed mode.  FP64 values: 6 per entry; FP32 values: 8 per entry (6 and two zeros), read as two
// float4.
template <typename T>
__device__ __forceinline__ void g_entry(const T* __restrict__ Gv, long long e, T g[6]);
template <>
__device__ __forceinline__ void g_entry<double>(const double* __restrict__ Gv, long long e, double g[6]) {
  // 6 doubles = 48 bytes per entry: every entry starts on a 16-byte boundary
  const double2* v = reinterpret_cast<const double2*>(Gv + e * 6);
  const double2 a = __ldg(v), b = __ldg(v + 1), c = __ldg(v + 2);
  g[0] = a.x; g[1] = a.y; g[2] = b.x; g[3] = b.y; g[4] = c.x; g[5] = c.y;
}
template <>
__device__ __forceinline__ void g_entry<float>(const float* __restrict__ Gv, long long e, float g[6]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(Gv) + 2 * e);
  const float4 b = __ldg(reinterpret_cast<const float4*>(Gv) + 2 * e + 1);
  g[0] = a.x; g[1] = a.y; g[2] = a.z; g[3] = a.w; g[4] = b.x; g[5] = b.y;
}

// entries per thread with their loads in flight together (FP32 / FP64 values)
template <typename T>
constexpr int g_batch() { return sizeof(T) == 4 ? 4 : 2; }
template <typename T>
__global__ void __launch_bounds__(256, 4) k_G_csr(DevMesh M, const T* __restrict__ Gv, const double* __restrict__ x,
                                                  double* gx, double scale, float* gx32 = nullptr) {
  __shared__ double red[6 * 32];
  const int p = blockIdx.x;
  const long long e0 = M.gp_ptr[p], e1 = M.gp_ptr[p + 1];
  T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  // a thread's entries e0 + tid + k blockDim in k order, g_batch<T>() of them with all their
  // loads in flight together (the row index, then x at the row, is a chain of two dependent loads)
  constexpr int kGU = g_batch<T>();
  const long long bd = blockDim.x;
  for (long long eb = e0 + threadIdx.x; eb < e1; eb += kGU * bd) {
    int row[kGU];
#pragma unroll
    for (int k = 0; k < kGU; ++k) row[k] = eb + k * bd < e1 ? __ldg(M.gp_row + eb + k * bd) : -1;
    T g[kGU][6];
#pragma unroll
    for (int k = 0; k < kGU; ++k)
      if (row[k] >= 0) g_entry<T>(Gv, eb + k * bd, g[k]);
    T v[kGU];
#pragma unroll
    for (int k = 0; k < kGU; ++k) v[k] = row[k] >= 0 ? T(__ldg(x + row[k])) : T(0);
#pragma unroll
    for (int k = 0; k < kGU; ++k)
      if (row[k] >= 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += g[k][c] * v[k];
  }
  double s[6];
  if constexpr (sizeof(T) == 4) {
    // the FP32 instance sums its block in FP32 (the FP64 pipe is narrow), in the order of
    // block_reduce_sum6, and rounds the sums to FP64 at the end
    block_reduce_sum6f(acc, reinterpret_cast<float*>(red));
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c] = double(acc[c]);
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c] = double(acc[c]);
    block_reduce_sum6(s, red);
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      gx[6 * (long long)p + c] = scale * s[c];
      if (gx32) gx32[6 * (long long)p + c] = (float)(scale * s[c]);
    }
}

// out[row] = ax * x[row] + bh * (G^T h)[row]   (x nullable); T as in k_G_csr.
template <typename T>
__global__ void k_GT_csr(DevMesh M, const T* __restrict__ GTv, const double* __restrict__ x, double ax,
                         const double* __restrict__ h, double bh, double* out) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row >= M.n_mult) return;
  double s = 0.0;
  for (long long e = M.gt_ptr[row]; e < M.gt_ptr[row + 1]; ++e) {
    const double* hq = h + 6 * (long long)M.gt_p[e];
    T g[6];
    g_entry<T>(GTv, e, g);
    double hv[6];
    if (sizeof(T) == 8) {
      const double2* h2 = reinterpret_cast<const double2*>(hq);
      const double2 a = __ldg(h2), b = __ldg(h2 + 1), c = __ldg(h2 + 2);
      hv[0] = a.x; hv[1] = a.y; hv[2] = b.x; hv[3] = b.y; hv[4] = c.x; hv[5] = c.y;
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) hv[c] = hq[c];
    }
    T t = T(0);
#pragma unroll
    for (int c = 0; c < 6; ++c) t += g[c] * T(hv[c]);
    s += double(t);
  }
  out[row] = (x ? ax * x[row] : 0.0) + bh * s;
}

// FP32: out[row] = x[row] - (G^T h)[row] with the padded FP32 values and h8, the FP32
// copy of h padded to 8 per subdomain (two float4 per entry and subdomain).
__global__ void k_GT_csr32(DevMesh M, const float* __restrict__ GTv8, const double* __restrict__ x,
                           const float* __restrict__ h8, double* out) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row >= M.n_mult) return;
  const long long e0 = M.gt_ptr[row], e1 = M.gt_ptr[row + 1];
  const float4* g4 = reinterpret_cast<const float4*>(GTv8);
  const float4* h4 = reinterpret_cast<const float4*>(h8);
  double s = 0.0;
  for (long long e = e0; e < e1; ++e) {
    const int q = __ldg(M.gt_p + e);
    const float4 a = __ldg(g4 + 2 * e), b = __ldg(g4 + 2 * e + 1);
    const float4 u = __ldg(h4 + 2 * q), v = __ldg(h4 + 2 * q + 1);
    const float t = a.x * u.x + a.y * u.y + a.z * u.z + a.w * u.w + b.x * v.x + b.y * v.y;
    s += double(t);
  }
  out[row] = x[row] - s;
}

constexpr int kGemvRows = 8;   // rows per 512-thread block of the coarse GEMVs (two warps per row)
constexpr int kGemv32B = 4;    // float4 loads per lane in flight in the FP32 coarse GEMV

// y = H x with the FP32 copy of H (n x n, rows padded with zeros to ld, a multiple of 4),
// x rounded to FP32 in shared memory; writes y (FP64) and its padded FP32 copy h8.  Two warps
// per row (kGemvRows rows per 512-thread block), each taking every other 32-float4 segment of
// the row, so that a lane has about a dozen float4 loads in flight at 64^3; the two halves are
// added in warp order.
__global__ void __launch_bounds__(512, 3) k_gemv32(const float* __restrict__ A, long long n, long long ld,
                                                   const double* __restrict__ x, const float* __restrict__ x32,
                                                   double* y, float* h8) {
  extern __shared__ __align__(16) float xs[];
  __shared__ float half[16];
  // x rounded to FP32: from x32 when the producer wrote that copy (no FP64 conversions here)
  for (long long j = threadIdx.x; j < ld; j += blockDim.x) xs[j] = j < n ? (x32 ? x32[j] : float(x[j])) : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long row = blockIdx.x * (long long)kGemvRows + (warp >> 1);
  const int hf = warp & 1;
  float acc = 0.f;
  if (row < n) {
    const long long n4 = ld >> 2;
    const float4* x4 = reinterpret_cast<const float4*>(xs);
    const float4* a4 = reinterpret_cast<const float4*>(A + row * ld);
    for (long long j0 = 32 * hf + lane; j0 < n4; j0 += 64 * kGemv32B) {
      float4 a[kGemv32B];   // the batch's loads issued before their products are summed
#pragma unroll
      for (int u = 0; u < kGemv32B; ++u) {
        const long long j = j0 + 64 * u;
        a[u] = j < n4 ? __ldg(a4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kGemv32B; ++u) {
        const long long j = j0 + 64 * u;
        if (j < n4) {
          const float4 v = x4[j];
          acc += a[u].x * v.x + a[u].y * v.y + a[u].z * v.z + a[u].w * v.w;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  }
  if (lane == 0) half[warp] = acc;
  __syncthreads();
  if (hf == 0 && lane == 0 && row < n) {
    const float t = half[warp] + half[warp + 1];
    y[row] = double(t);
    h8[(row / 6) * 8 + row % 6] = t;
  }
}

// Entry values of G: e' runs over the row-ordered entries, e = gt_e[e'] is the same
// entry in subdomain order (a permutation), v = coef * R_p[slot dof][c].
__global__ void k_fill_G(DevMesh M, const int* __restrict__ gp_slot, const double* __restrict__ gp_coef,
                         const int* __restrict__ gt_e, double* Gv, float* Gv32, double* GTv, float* GTv32) {
  const long long et = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (et >= M.n_gpairs) return;
  const long long e = gt_e[et];
  const long long slot = gp_slot[e];
  const SubDev& S = M.subs[M.slot_sub[slot]];
  const double* r = M.R + S.r_off + (long long)M.slot_ldof[slot] * 6;
  const double cf = gp_coef[e];
  for (int c = 0; c < 8; ++c) {
    const double v = c < 6 ? cf * r[c] : 0.0;
    if (c < 6) {
      Gv[e * 6 + c] = v;
      GTv[et * 6 + c] = v;
    }
    Gv32[e * 8 + c] = (float)v;
    GTv32[et * 8 + c] = (float)v;
  }
}

// out = v + R_p alpha_p on the dofs of subdomain p = blockIdx.y.
__global__ void k_add_R_alpha(DevMesh M, const double* __restrict__ v, const double* __restrict__ alpha,
                              double* out) {
  const SubDev& S = M.subs[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n_dof) return;
  const double* r = M.R + S.r_off + (long long)i * 6;
  const double* al = alpha + 6 * (long long)blockIdx.y;
  double s = v[S.dof_off + i];
#pragma unroll
  for (int c = 0; c < 6; ++c) s += r[c] * al[c];
  out[S.dof_off + i] = s;
}

// y = alpha * A x, A dense n x n row-major FP64.  Two warps per row (kGemvRows rows per
// 512-thread block), each taking every other 32-double2 segment of the row (16-byte loads: n is
// even, 6 coarse unknowns per subdomain) with kGemv64B of its loads issued before their products
// are summed; the halves are added in warp order.
constexpr int kGemv64B = 6;
__global__ void __launch_bounds__(512, 3) k_gemv64(const double* __restrict__ A, long long n,
                                                   const double* __restrict__ x, double alpha, double* y) {
  __shared__ double half[16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long row = blockIdx.x * (long long)kGemvRows + (warp >> 1);
  const int hf = warp & 1;
  double acc = 0.0;
  if (row < n) {
    const long long n2 = n >> 1;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    const double2* a2 = reinterpret_cast<const double2*>(A + row * n);
    for (long long j0 = 32 * hf + lane; j0 < n2; j0 += 64 * kGemv64B) {
      double2 a[kGemv64B];
#pragma unroll
      for (int u = 0; u < kGemv64B; ++u) {
        const long long j = j0 + 64 * u;
        a[u] = j < n2 ? __ldg(a2 + j) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < kGemv64B; ++u) {
        const long long j = j0 + 64 * u;
        if (j < n2) {
          const double2 v = __ldg(x2 + j);
          acc += a[u].x * v.x + a[u].y * v.y;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  }
  if (lane == 0) half[warp] = acc;
  __syncthreads();
  if (hf == 0 && lane == 0 && row < n) y[row] = alpha * (half[warp] + half[warp + 1]);
}

// Lumped preconditioner, subdomain part: v = K_bb (B^T w) on the interface slots.
// K_bb comes from the subdomain's boundary blocks (kbb + kbb_off[p]): its shape's
// elastic template or its own blocks when it has plastic points.
// T: FP64 blocks, or their FP32 copy for the inner iterations of the mixed mode.
constexpr int kXU = 4;       // copy slots per thread with their B^T gathers in flight together
// stencil neighbours per batch of block loads in the lumped apply (FP32 / FP64 blocks)
template <typename T>
constexpr int nb_batch() { return sizeof(T) == 4 ? 9 : 3; }
template <typename T>
__global__ void __launch_bounds__(256, 4) k_lumped(DevMesh M, const double* __restrict__ w, const T* __restrict__ kbb,
                                                   const long long* __restrict__ kbb_off, double* cbuf) {
  extern __shared__ __align__(16) unsigned char xs_raw[];
  T* xs = reinterpret_cast<T*>(xs_raw);
  const int p = blockIdx.x;
  const SubDev S = M.subs[p];
  for (int s0 = threadIdx.x; s0 < S.n_copy; s0 += kXU * blockDim.x) {
    long long sl[kXU];
    double v[kXU];
#pragma unroll
    for (int k = 0; k < kXU; ++k) sl[k] = s0 + k * (int)blockDim.x < S.n_copy ? S.copy_off + s0 + k * blockDim.x : -1;
    bt_at_slots<kXU>(M, w, sl, v);
#pragma unroll
    for (int k = 0; k < kXU; ++k)
      if (sl[k] >= 0) xs[s0 + k * blockDim.x] = T(v[k]);
  }
  __syncthreads();
  // blocks stored [t][cc][3 b + a] (neighbour t, column cc, row 3 b + a of boundary node b), all 27
  // neighbours present in the storage (zero where the stencil has none); the neighbours are
  // visited in order, nb_batch<T>() of them with their slot and block loads issued together
  const T* kb = kbb + kbb_off[p];
  const long long nr = 3LL * S.n_bnd;
  for (int q = threadIdx.x; q < S.n_copy; q += blockDim.x) {
    const long long slot = S.copy_off + q;
    const int b = M.slot_bnd[slot], a = q % 3;
    const T* kv = kb + 3LL * b + a;
    const int* nbp = M.sub_nbr + (slot / 3) * 28;
    T s = T(0);
    constexpr int NB = nb_batch<T>();
#pragma unroll
    for (int t0 = 0; t0 < 27; t0 += NB) {
      int nb[NB];
      T k0[NB], k1[NB], k2[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int t = t0 + u;
        nb[u] = __ldg(nbp + t);
        k0[u] = __ldg(kv + (3 * t) * nr);
        k1[u] = __ldg(kv + (3 * t + 1) * nr);
        k2[u] = __ldg(kv + (3 * t + 2) * nr);
      }
#pragma unroll
      for (int u = 0; u < NB; ++u)
        if (nb[u] >= 0) {
          const int lb = (int)(nb[u] - S.copy_off);
          s += k0[u] * xs[lb] + k1[u] * xs[lb + 1] + k2[u] * xs[lb + 2];
        }
    }
    cbuf[slot] = double(s);
  }
}

// Dirichlet preconditioner: B^T w onto the copy-slot dofs of the full local vectors.
__global__ void k_slots_to_full(DevMesh M, const double* __restrict__ w, double* xfull) {
  const long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (sl >= M.n_copy) return;
  const SubDev& S = M.subs[M.slot_sub[sl]];
  xfull[S.dof_off + M.slot_ldof[sl]] = bt_at_slot(M, w, sl);
}

__global__ void k_slots_diff(DevMesh M, const double* __restrict__ v, const double* __restrict__ t, double* cbuf) {
  const long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (sl >= M.n_copy) return;
  const long long d = M.subs[M.slot_sub[sl]].dof_off + M.slot_ldof[sl];
  cbuf[sl] = v[d] - t[d];
}

// Deterministic dot product: fixed grid, fixed per-block order, fixed final order.
__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, long long n,
                              double* partial) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  s = block_reduce_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_dot_final(const double* partial, int nparts, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
  s = block_reduce_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (x ? a * x[i] : 0.0) + (y ? b * y[i] : 0.0);
}

// Scalars: sc[0] = y.w (current), sc[1] = y.w (previous), sc[2] = p.Fp, sc[3] = w.w,
// sc[4] = beta, sc[5] = gamma, sc[6] = breakdown flag.
__global__ void k_p_update(long long n, const double* __restrict__ y, double* p, const double* sc, int first) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double beta = first ? 0.0 : sc[0] / sc[1];
  p[i] = first ? y[i] : y[i] + beta * p[i];
}

__global__ void k_lam_r_update(long long n, const double* __restrict__ p, const double* __restrict__ Fp, double* lam,
                               double* r, const double* sc) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gamma = sc[0] / sc[2];
  lam[i] += gamma * p[i];
  r[i] -= gamma * Fp[i];
}

__global__ void k_scalars_after_pfp(double* sc) {
  if (threadIdx.x == 0) {
    sc[5] = sc[0] / sc[2];
    if (!(sc[2] > 0.0)) sc[6] = 1.0;
  }
}

// ---------------------------------------------------------------------------
// Device-side control of the graph-driven PCGP (Algorithm 3 scalars).  The loop
// body ends with k_pcg_post, which sets the WHILE condition of the graph: it
// continues until the stop test of the last iteration held, the iteration limit
// is reached, a breakdown or a non-finite value was met, or the body has run
// 2 maxit + 4 times (a hard bound on the device loop).
// ---------------------------------------------------------------------------
__global__ void k_pcg_init(double* sc, double tol2, int maxit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc[kDone] = 0.0;
    sc[kStatus] = 0.0;
    sc[kStopAfter] = 0.0;
    sc[kFirst] = 1.0;
    sc[kTol2] = tol2;
    sc[kIter] = 0.0;
    sc[kMaxit] = (double)maxit;
    sc[kLastWW] = 0.0;
    sc[kBodyRuns] = 0.0;
  }
}

__global__ void k_dot2_partial(const double* __restrict__ x1, const double* __restrict__ y1,
                               const double* __restrict__ x2, const double* __restrict__ y2, long long n,
                               double* partial) {
  __shared__ double red[32];
  double s1 = 0.0, s2 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    s1 += x1[i] * y1[i];
    s2 += x2[i] * y2[i];
  }
  s1 = block_reduce_sum(s1, red);
  s2 = block_reduce_sum(s2, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s1;
    partial[gridDim.x + blockIdx.x] = s2;
  }
}

__global__ void k_dot2_final(const double* partial, int nparts, double* out1, double* out2) {
  __shared__ double red[32];
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    s1 += partial[i];
    s2 += partial[nparts + i];
  }
  s1 = block_reduce_sum(s1, red);
  s2 = block_reduce_sum(s2, red);
  if (threadIdx.x == 0) {
    *out1 = s1;
    *out2 = s2;
  }
}

__global__ void k_pcg_pre(double* sc) {
  if (threadIdx.x || blockIdx.x) return;
  pcg_pre_logic(sc);
}

__global__ void k_pcg_mid(double* sc) {
  if (threadIdx.x || blockIdx.x) return;
  pcg_mid_logic(sc);
}

__global__ void k_pcg_post(double* sc, cudaGraphConditionalHandle h) {
  if (threadIdx.x || blockIdx.x) return;
  const bool more = pcg_post_logic(sc);
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Fused kernels of the graph-driven inner PCGP iteration.  Each folds a dot product
// (and the scalar step that follows it) into the kernel that produces the vector:
// every block writes its partial sum, and the block that arrives last (counted with
// one atomic per block) sums the partials in block order, so the result is the same
// whichever block finishes last; that block resets its counter for the next launch.
// The grid is fixed (kFusedBlocks, grid-stride loops), which fixes the summation order.
// ---------------------------------------------------------------------------
__device__ bool grid_sum_last(double s, double* partial, int* ctr, double* red, double* total) {
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    __threadfence();
    is_last = atomicAdd(ctr, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(partial + i);
  t = block_reduce_sum(t, red);
  if (threadIdx.x == 0) {
    *total = t;
    *ctr = 0;
  }
  return true;   // *total valid in thread 0
}

// out = x - G^T h (FP32 padded values, h8 the padded FP32 coarse vector) with the fused
// dot: mode 0 -> sc[kWW] = out.out (w = P r); mode 1 -> sc[kYW] = out.v (y = P z, v = w),
// then the stop test of the iteration (pcg_pre), and with deflation (k = sc[kDeflK] > 0)
// also d_j = out.AW_j and mu = E^-1 d -> sc[kMu0 + i].  The partial sums of value j sit at
// partial[j * gridDim.x + block].  kDefl: the instance that carries the deflation sums (AW given).
template <bool kDefl>
__global__ void __launch_bounds__(256, 4)
    k_GT32_dot(DevMesh M, const float* __restrict__ GTv8, const double* __restrict__ x, const float* __restrict__ h8,
               double* out, const double* __restrict__ v, int mode, double* sc, double* partial, int* ctr,
               const double* __restrict__ AW, const double* __restrict__ Einv) {
  __shared__ double red[32];
  __shared__ int is_last;
  const float4* g4 = reinterpret_cast<const float4*>(GTv8);
  const float4* h4 = reinterpret_cast<const float4*>(h8);
  const int kd = (kDefl && mode == 1 && AW) ? (int)sc[kDeflK] : 0;
  const long long m = M.n_mult;
  constexpr int KD = kDefl ? kDeflMax : 1;
  double acc = 0.0, accd[KD];
#pragma unroll
  for (int j = 0; j < KD; ++j) accd[j] = 0.0;
  // a thread's rows row0 + i stride in i order, two at a time with their loads interleaved
  // (row range, then the entries' subdomains, then h at those: three dependent loads)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; row0 < m; row0 += 2 * stride) {
    const long long row1 = row0 + stride;
    const bool has1 = row1 < m;
    const long long e0 = M.gt_ptr[row0], e1 = M.gt_ptr[row0 + 1];
    const long long f0 = has1 ? M.gt_ptr[row1] : 0, f1 = has1 ? M.gt_ptr[row1 + 1] : 0;
    const double x0 = x[row0], x1 = has1 ? x[row1] : 0.0;
    const double v0 = mode == 0 ? 0.0 : v[row0], v1 = (mode == 0 || !has1) ? 0.0 : v[row1];
    float s0 = 0.f, s1 = 0.f;   // a row's few FP32 products summed in FP32
    for (long long k = 0; e0 + k < e1 || f0 + k < f1; ++k) {
      const bool a0 = e0 + k < e1, a1 = f0 + k < f1;
      int q0 = 0, q1 = 0;
      float4 ga0, gb0, ga1, gb1;
      if (a0) {
        q0 = __ldg(M.gt_p + e0 + k);
        ga0 = __ldg(g4 + 2 * (e0 + k));
        gb0 = __ldg(g4 + 2 * (e0 + k) + 1);
      }
      if (a1) {
        q1 = __ldg(M.gt_p + f0 + k);
        ga1 = __ldg(g4 + 2 * (f0 + k));
        gb1 = __ldg(g4 + 2 * (f0 + k) + 1);
      }
      if (a0) {
        const float4 u = __ldg(h4 + 2 * q0), w = __ldg(h4 + 2 * q0 + 1);
        s0 += ga0.x * u.x + ga0.y * u.y + ga0.z * u.z + ga0.w * u.w + gb0.x * w.x + gb0.y * w.y;
      }
      if (a1) {
        const float4 u = __ldg(h4 + 2 * q1), w = __ldg(h4 + 2 * q1 + 1);
        s1 += ga1.x * u.x + ga1.y * u.y + ga1.z * u.z + ga1.w * u.w + gb1.x * w.x + gb1.y * w.y;
      }
    }
    const double o0 = x0 - double(s0);
    out[row0] = o0;
    acc += o0 * (mode == 0 ? o0 : v0);
    if constexpr (kDefl) {
#pragma unroll
      for (int j = 0; j < KD; ++j)
        if (j < kd) accd[j] += o0 * AW[(long long)j * m + row0];
    }
    if (has1) {
      const double o1 = x1 - double(s1);
      out[row1] = o1;
      acc += o1 * (mode == 0 ? o1 : v1);
      if constexpr (kDefl) {
#pragma unroll
        for (int j = 0; j < KD; ++j)
          if (j < kd) accd[j] += o1 * AW[(long long)j * m + row1];
      }
    }
  }
  acc = block_reduce_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  for (int j = 0; j < kd && j < KD; ++j) {
    const double t = block_reduce_sum(accd[j], red);
    if (threadIdx.x == 0) partial[(long long)(1 + j) * gridDim.x + blockIdx.x] = t;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(ctr, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double tot[1 + KD];
  for (int j = 0; j <= kd && j <= KD; ++j) {
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(partial + (long long)j * gridDim.x + i);
    tot[j] = block_reduce_sum(t, red);
  }
  if (threadIdx.x == 0) {
    *ctr = 0;
    if (mode == 0) {
      sc[kWW] = tot[0];
    } else {
      sc[kYW] = tot[0];
      pcg_pre_logic(sc);
      for (int i = 0; i < kd; ++i) {
        double mu = 0.0;
        for (int j = 0; j < kd; ++j) mu += Einv[i * kDeflMax + j] * tot[1 + j];
        sc[kMu0 + i] = mu;
      }
    }
  }
}

// Fp = B cbuf with the fused dot sc[kPFP] = p.Fp, then the breakdown test (pcg_mid).
__global__ void k_contract_dot(DevMesh M, const double* __restrict__ cbuf, double* Fp, const double* __restrict__ p,
                               double* sc, double* partial, int* ctr) {
  __shared__ double red[32];
  double acc = 0.0;
  // a thread's rows in order, two at a time (their gathers from cbuf overlap)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; row0 < M.n_mult; row0 += 2 * stride) {
    const long long row1 = row0 + stride;
    const bool has1 = row1 < M.n_mult;
    const double p0 = p[row0], p1 = has1 ? p[row1] : 0.0;
    const double y0 = b_at_row(M, cbuf, row0);
    const double y1 = has1 ? b_at_row(M, cbuf, row1) : 0.0;
    Fp[row0] = y0;
    acc += p0 * y0;
    if (has1) {
      Fp[row1] = y1;
      acc += p1 * y1;
    }
  }
  acc = block_reduce_sum(acc, red);
  double tot = 0.0;
  if (grid_sum_last(acc, partial, ctr, red, &tot) && threadIdx.x == 0) {
    sc[kPFP] = tot;
    pcg_mid_logic(sc);
  }
}

// lam += gamma p, r -= gamma Fp (no-op once done); the last block closes the body run
// (pcg_post) and, inside a graph (has_h), sets the WHILE condition.
__global__ void k_lam_r_update_post(long long n, const double* __restrict__ p, const double* __restrict__ Fp,
                                    double* lam, double* r, double* sc, int* ctr, cudaGraphConditionalHandle h,
                                    int has_h) {
  __shared__ int is_last;
  __shared__ double s_gamma;
  const bool done = sc[kDone] != 0.0;
  if (!done) {
    // one FP64 division per block (the FP64 pipe is narrow): gamma for all its threads
    if (threadIdx.x == 0) s_gamma = sc[kYW] / sc[kPFP];
    __syncthreads();
    const double gamma = s_gamma;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
      const long long i1 = i + stride;
      const bool has1 = i1 < n;
      const double l0 = lam[i], p0 = p[i], r0 = r[i], f0 = Fp[i];
      const double l1 = has1 ? lam[i1] : 0.0, p1 = has1 ? p[i1] : 0.0, r1 = has1 ? r[i1] : 0.0,
                   f1 = has1 ? Fp[i1] : 0.0;
      lam[i] = l0 + gamma * p0;
      r[i] = r0 - gamma * f0;
      if (has1) {
        lam[i1] = l1 + gamma * p1;
        r[i1] = r1 - gamma * f1;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(ctr, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    *ctr = 0;
    const bool more = pcg_post_logic(sc);
    if (has_h) cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

__global__ void k_p_update_g(long long n, const double* __restrict__ y, double* p, const double* sc,
                             const double* __restrict__ W) {
  __shared__ double s_beta;
  if (sc[kDone] != 0.0) return;   // the same for every thread
  const bool first = sc[kFirst] != 0.0;
  if (threadIdx.x == 0) s_beta = first ? 0.0 : sc[kYW] / sc[kYWPrev];   // one division per block
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double beta = s_beta;
  double v = first ? y[i] : y[i] + beta * p[i];
  if (W) {   // deflated direction: p = y + beta p - W mu
    const int kd = (int)sc[kDeflK];
    for (int j = 0; j < kd; ++j) v -= sc[kMu0 + j] * W[(long long)j * n + i];
  }
  p[i] = v;
}

__global__ void k_lam_r_update_g(long long n, const double* __restrict__ p, const double* __restrict__ Fp,
                                 double* lam, double* r, const double* sc) {
  __shared__ double s_gamma;
  if (sc[kDone] != 0.0) return;   // the same for every thread
  if (threadIdx.x == 0) s_gamma = sc[kYW] / sc[kPFP];   // one division per block
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gamma = s_gamma;
  lam[i] += gamma * p[i];
  r[i] -= gamma * Fp[i];
}

// ---------------------------------------------------------------------------
// Coarse matrix G G^T = R^T B^T B R assembled per subdomain pair (p >= q):
// block[a][b] = sum over groups with copies i in p and j in q of
// R_p[slot_i][a] (sum_rows B[row][i] B[row][j]) R_q[slot_j][b].
// ---------------------------------------------------------------------------
__global__ void k_coarse_assemble(DevMesh M, const int* __restrict__ pair_p, const int* __restrict__ pair_q,
                                  const long long* __restrict__ pair_start, const int* __restrict__ trip_group,
                                  const int* __restrict__ trip_i, const int* __restrict__ trip_j, long long n_pairs,
                                  double* A, long long l) {
  const long long pr = blockIdx.x;
  if (pr >= n_pairs) return;
  const int e = threadIdx.x;
  if (e >= 36) return;
  const int a = e / 6, b = e % 6;
  const int p = pair_p[pr], q = pair_q[pr];
  const double* Rp = M.R + M.subs[p].r_off;
  const double* Rq = M.R + M.subs[q].r_off;
  double s = 0.0;
  for (long long t = pair_start[pr]; t < pair_start[pr + 1]; ++t) {
    const GroupDev& g = M.groups[trip_group[t]];
    const int i = trip_i[t], j = trip_j[t];
    double m;
    if (g.dirichlet) {
      m = (i == j) ? 1.0 : 0.0;
    } else {
      m = 0.0;
      for (int r = 1; r < g.k; ++r) m += M.helm[r * 8 + i] * M.helm[r * 8 + j];
    }
    s += Rp[(long long)M.slot_ldof[g.slot[i]] * 6 + a] * m * Rq[(long long)M.slot_ldof[g.slot[j]] * 6 + b];
  }
  A[(6LL * p + a) * l + 6LL * q + b] = s;
  if (p != q) A[(6LL * q + b) * l + 6LL * p + a] = s;
}

// The same blocks into the block-tridiagonal storage of the plane solver: subdomain p lies in
// plane p / per_plane at local index p % per_plane; Adiag[k] (n_pl x n_pl, both triangles) and
// Aoff[k] = the block of plane k's rows and plane k-1's columns (p >= q puts q's plane at or
// below p's, and neighbours differ by at most one plane).
__global__ void k_coarse_assemble_planes(DevMesh M, const int* __restrict__ pair_p, const int* __restrict__ pair_q,
                                         const long long* __restrict__ pair_start, const int* __restrict__ trip_group,
                                         const int* __restrict__ trip_i, const int* __restrict__ trip_j,
                                         long long n_pairs, double* Adiag, double* Aoff, int per_plane, int n_pl) {
  const long long pr = blockIdx.x;
  if (pr >= n_pairs) return;
  const int e = threadIdx.x;
  if (e >= 36) return;
  const int a = e / 6, b = e % 6;
  const int p = pair_p[pr], q = pair_q[pr];
  const double* Rp = M.R + M.subs[p].r_off;
  const double* Rq = M.R + M.subs[q].r_off;
  double s = 0.0;
  for (long long t = pair_start[pr]; t < pair_start[pr + 1]; ++t) {
    const GroupDev& g = M.groups[trip_group[t]];
    const int i = trip_i[t], j = trip_j[t];
    double m;
    if (g.dirichlet) {
      m = (i == j) ? 1.0 : 0.0;
    } else {
      m = 0.0;
      for (int r = 1; r < g.k; ++r) m += M.helm[r * 8 + i] * M.helm[r * 8 + j];
    }
    s += Rp[(long long)M.slot_ldof[g.slot[i]] * 6 + a] * m * Rq[(long long)M.slot_ldof[g.slot[j]] * 6 + b];
  }
  const int kp = p / per_plane, kq = q / per_plane;
  const long long ip = 6LL * (p % per_plane) + a, iq = 6LL * (q % per_plane) + b;
  const long long blk = (long long)n_pl * n_pl;
  if (kp == kq) {
    Adiag[kp * blk + ip * n_pl + iq] = s;
    if (p != q) Adiag[kp * blk + iq * n_pl + ip] = s;
  } else {
    Aoff[kp * blk + ip * n_pl + iq] = s;   // kq = kp - 1
  }
}

// Apply of the plane solver (H = (G G^T)^-1 by block LDL^T over the planes):
// first y_k = alpha W_k x_k for every plane (blockIdx.y = k), then the forward steps
// y_k -= V_k y_{k-1}, k = 1..np-1, and the backward steps y_k -= U_k y_{k+1}, k = np-2..0.
// Two warps per row, the other plane's segment staged in shared memory.  T: FP64 blocks, or
// their FP32 copies (FP32 products and sums); y8 (nullable): the padded FP32 copy of the final
// y written by the last step that touches a plane (final != 0).
// Rows of a plane block: kPlaneRows rows per 256-thread CTA, two warps per row, each lane
// keeping four 16- or 8-byte loads in flight; the two warps' sums meet in shared memory.
constexpr int kPlaneRows = 4;

template <typename T>
__device__ __forceinline__ double plane_part_dot(const T* __restrict__ row, const void* xs, int n, int sub);
template <>
__device__ __forceinline__ double plane_part_dot<double>(const double* __restrict__ row, const void* xs, int n,
                                                         int sub) {
  const double2* r2 = reinterpret_cast<const double2*>(row);
  const double2* x2 = reinterpret_cast<const double2*>(xs);
  double acc = 0.0;
#pragma unroll 4
  for (int j = sub; j < (n >> 1); j += 64) {
    const double2 a = __ldg(r2 + j), v = x2[j];
    acc += a.x * v.x + a.y * v.y;
  }
  return acc;
}
template <>
__device__ __forceinline__ double plane_part_dot<float>(const float* __restrict__ row, const void* xs, int n, int sub) {
  const float2* r2 = reinterpret_cast<const float2*>(row);
  const float2* x2 = reinterpret_cast<const float2*>(xs);
  float acc = 0.f;
#pragma unroll 4
  for (int j = sub; j < (n >> 1); j += 64) {
    const float2 a = __ldg(r2 + j), v = x2[j];
    acc += a.x * v.x + a.y * v.y;
  }
  return double(acc);
}

// Row r of this CTA (r < kPlaneRows) of matrix rows `rows` (n wide): the dot with the staged x,
// valid in thread (r * 64) of the CTA.
template <typename T>
__device__ __forceinline__ double plane_row_dot(const T* __restrict__ rowp, const void* xs, int n, double* red) {
  const int sub = threadIdx.x & 63, pair = threadIdx.x >> 6, lane = threadIdx.x & 31;
  double acc = rowp ? plane_part_dot<T>(rowp, xs, n, sub) : 0.0;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0 && sub >= 32) red[pair] = acc;
  __syncthreads();
  if (sub == 0) acc += red[pair];
  return acc;
}

template <typename T>
__device__ __forceinline__ void plane_stage(const double* __restrict__ x, int n, void* xs) {
  T* t = reinterpret_cast<T*>(xs);
  for (int j = threadIdx.x; j < n; j += blockDim.x) t[j] = T(x[j]);
  __syncthreads();
}

__device__ __forceinline__ void plane_y8(float* y8, long long grow, double v) {
  if (y8) y8[(grow / 6) * 8 + grow % 6] = float(v);
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_first(const T* __restrict__ W, int n, const double* __restrict__ x,
                                                     double alpha, double* y, float* y8, int final) {
  extern __shared__ __align__(16) unsigned char plane_xs[];
  __shared__ double red[kPlaneRows];
  const int k = blockIdx.y;
  plane_stage<T>(x + (long long)k * n, n, plane_xs);
  const int r = blockIdx.x * kPlaneRows + (threadIdx.x >> 6);
  const double d = plane_row_dot<T>(r < n ? W + ((long long)k * n + r) * n : nullptr, plane_xs, n, red);
  if ((threadIdx.x & 63) == 0 && r < n) {
    const long long g = (long long)k * n + r;
    const double v = alpha * d;
    y[g] = v;
    if (final) plane_y8(y8, g, v);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_step(const T* __restrict__ Mk, int n, const double* __restrict__ y_other,
                                                    double* y_k, long long row0, float* y8, int final) {
  extern __shared__ __align__(16) unsigned char plane_xs[];
  __shared__ double red[kPlaneRows];
  plane_stage<T>(y_other, n, plane_xs);
  const int r = blockIdx.x * kPlaneRows + (threadIdx.x >> 6);
  const double d = plane_row_dot<T>(r < n ? Mk + (long long)r * n : nullptr, plane_xs, n, red);
  if ((threadIdx.x & 63) == 0 && r < n) {
    const double v = y_k[r] - d;
    y_k[r] = v;
    if (final) plane_y8(y8, row0 + r, v);
  }
}

// ---------------------------------------------------------------------------
// Dense FP64 building blocks for the coarse problem (set-up only).
// ---------------------------------------------------------------------------
constexpr int kD = 32;

// Factor the kD x kD diagonal block at (k0,k0) of A in place (lower) and write
// its inverse to Dinv (kD x kD).  One warp.
__global__ void k_dense_diag(double* A, long long l, long long k0, int jb, double* Dinv, int* err) {
  __shared__ double D[kD][kD + 1];
  __shared__ double X[kD][kD + 1];
  const int lane = threadIdx.x;
  for (int r = 0; r < jb; ++r)
    if (lane < jb) D[r][lane] = lane <= r ? A[(k0 + r) * l + k0 + lane] : 0.0;
  __syncwarp();
  for (int c = 0; c < jb; ++c) {
    double d = D[c][c];
    if (!(d > 0.0)) {
      if (lane == 0) atomicOr(err, 1);
      d = 1.0;
    }
    d = sqrt(d);
    const double inv = 1.0 / d;
    __syncwarp();
    if (lane == c) D[c][c] = d;
    if (lane > c && lane < jb) D[lane][c] *= inv;
    __syncwarp();
    if (lane > c && lane < jb) {
      const double lrc = D[lane][c];
      for (int s = c + 1; s <= lane; ++s) D[lane][s] -= lrc * D[s][c];
    }
    __syncwarp();
  }
  if (lane < jb) {
    const int s = lane;
    for (int r = 0; r < jb; ++r) {
      if (r < s) {
        X[r][s] = 0.0;
      } else {
        double acc = (r == s) ? 1.0 : 0.0;
        for (int t = s; t < r; ++t) acc -= D[r][t] * X[t][s];
        X[r][s] = acc / D[r][r];
      }
    }
  }
  __syncwarp();
  for (int r = 0; r < jb; ++r)
    if (lane < jb) {
      A[(k0 + r) * l + k0 + lane] = lane <= r ? D[r][lane] : 0.0;
      Dinv[r * kD + lane] = X[r][lane];
    }
}

// Panel: A[i][k0+c] <- sum_{s<=c} A[i][k0+s] Dinv[c][s] for rows i >= k0+jb.  One warp per row.
__global__ void k_dense_panel(double* A, long long l, long long k0, int jb, const double* Dinv) {
  const long long i = k0 + jb + blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= l) return;
  double* row = A + i * l + k0;
  double val = 0.0;
  if (lane < jb)
    for (int s = 0; s <= lane; ++s) val += row[s] * Dinv[lane * kD + s];
  __syncwarp();
  if (lane < jb) row[lane] = val;
}

// Generic tiled FP64 GEMM: C[i][j] = beta C[i][j] + alpha sum_t A(i,t) B(t,j),
// A(i,t) = A[i*sai + t*sat], B(t,j) = B[t*sbt + j*sbj], t in [k_lo, k_hi).
// lower_only: skip tiles strictly above the diagonal and entries j > i.
// ktri: start t at max(tile row, tile col) (for Y^T Y with Y lower-triangular).
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) k_dgemm(long long Mr, long long Nc, long long k_lo, long long k_hi,
                                               double alpha, const double* __restrict__ A, long long sai,
                                               long long sat, const double* __restrict__ B, long long sbt,
                                               long long sbj, double beta, double* C, long long ldc, int lower_only,
                                               int ktri) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const long long i0 = blockIdx.y * (long long)TM, j0 = blockIdx.x * (long long)TN;
  if (lower_only && j0 > i0 + TM - 1) return;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  long long kbeg = k_lo;
  if (ktri) kbeg = i0 > j0 ? (i0 > k_lo ? i0 : k_lo) : (j0 > k_lo ? j0 : k_lo);
  for (long long kt = kbeg; kt < k_hi; kt += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      const int kk = e / TM, ii = e % TM;
      const long long gi = i0 + ii, gk = kt + kk;
      As[kk][ii] = (gi < Mr && gk < k_hi) ? A[gi * sai + gk * sat] : 0.0;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      const int kk = e / TN, jj = e % TN;
      const long long gj = j0 + jj, gk = kt + kk;
      Bs[kk][jj] = (gj < Nc && gk < k_hi) ? B[gk * sbt + gj * sbj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty * 4 + u];
        b[u] = Bs[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long gi = i0 + ty * 4 + u, gj = j0 + tx * 4 + v;
      if (gi < Mr && gj < Nc && (!lower_only || gj <= gi)) {
        double* c = C + gi * ldc + gj;
        *c = (beta == 0.0 ? 0.0 : beta * *c) + alpha * acc[u][v];
      }
    }
}

void dgemm(long long Mr, long long Nc, long long k_lo, long long k_hi, double alpha, const double* A, long long sai,
           long long sat, const double* B, long long sbt, long long sbj, double beta, double* C, long long ldc,
           int lower_only, int ktri, cudaStream_t st) {
  if (Mr <= 0 || Nc <= 0) return;
  dim3 grid((unsigned)((Nc + TN - 1) / TN), (unsigned)((Mr + TM - 1) / TM));
  k_dgemm<<<grid, 256, 0, st>>>(Mr, Nc, k_lo, k_hi, alpha, A, sai, sat, B, sbt, sbj, beta, C, ldc, lower_only, ktri);
}

}  // namespace

void launch_contract(const DevMesh& M, const double* cbuf, double* y, cudaStream_t st) {
  if (M.n_mult > 0) k_contract<<<blocks_for(M.n_mult, 256), 256, 0, st>>>(M, cbuf, y);
}

void launch_G_apply(const DevMesh& M, const double* x_lam, const double* x_full, double* gx, double scale,
                    cudaStream_t st) {
  if (x_lam) k_G_csr<double><<<M.n_sub, 256, 0, st>>>(M, M.Gv, x_lam, gx, scale);
  else k_G_full<<<M.n_sub, 256, 0, st>>>(M, x_full, gx, scale);
}

void launch_GT_update(const DevMesh& M, const double* x, double ax, const double* h, double bh, double* out,
                      cudaStream_t st) {
  if (M.n_mult > 0) k_GT_csr<double><<<blocks_for(M.n_mult, 256), 256, 0, st>>>(M, M.GTv, x, ax, h, bh, out);
}

void launch_fill_G(const DevMesh& M, const int* gp_slot, const double* gp_coef, const int* gt_e, double* Gv,
                   float* Gv32, double* GTv, float* GTv32, cudaStream_t st) {
  if (M.n_gpairs > 0)
    k_fill_G<<<blocks_for(M.n_gpairs, 256), 256, 0, st>>>(M, gp_slot, gp_coef, gt_e, Gv, Gv32, GTv, GTv32);
}

void launch_gemv(const double* A, long long n, const double* x, double alpha, double* y, cudaStream_t st) {
  if (n > 0) k_gemv64<<<blocks_for(n, kGemvRows), 512, 0, st>>>(A, n, x, alpha, y);
}

// FP32 copy of the dense H with rows padded to h32_ld(l) (zeros beyond column l).
__global__ void k_h_to_f32(const double* __restrict__ H, long long l, long long ld, float* H32) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= l * ld) return;
  const long long r = i / ld, c = i % ld;
  H32[i] = c < l ? float(H[r * l + c]) : 0.f;
}

void launch_h_to_f32(const double* H, long long l, float* H32, cudaStream_t st) {
  const long long ld = h32_ld(l);
  if (l > 0) k_h_to_f32<<<blocks_for(l * ld, 256), 256, 0, st>>>(H, l, ld, H32);
}

void launch_project32(const DevMesh& M, const CoarseOp& C, const double* x, double* gx, float* gx32, double* hx,
                      float* hx8, double* out, cudaStream_t st) {
  launch_G32_coarse32(M, C, x, gx, gx32, hx, hx8, st);
  if (M.n_mult > 0) k_GT_csr32<<<blocks_for(M.n_mult, 256), 256, 0, st>>>(M, M.GTv32, x, hx8, out);
}

void launch_add_R_alpha(const DevMesh& M, const double* v, const double* alpha, double* out, int max_ndof,
                       cudaStream_t st) {
  if (M.n_sub <= 0 || max_ndof <= 0) return;
  k_add_R_alpha<<<dim3((unsigned)((max_ndof + 255) / 256), (unsigned)M.n_sub), 256, 0, st>>>(M, v, alpha, out);
}

void launch_lumped(const DevMesh& M, const double* w, const double* kbb, const long long* kbb_off, double* cbuf,
                   cudaStream_t st, int max_copy) {
  const size_t smem = sizeof(double) * (size_t)(max_copy > 0 ? max_copy : 1);
  static const int lim = dyn_smem_limit((const void*)k_lumped<double>);
  cudaFuncSetAttribute(k_lumped<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  k_lumped<double><<<M.n_sub, 256, smem, st>>>(M, w, kbb, kbb_off, cbuf);
}

void launch_slots_to_full(const DevMesh& M, const double* w, double* xfull, cudaStream_t st) {
  if (M.n_copy > 0) k_slots_to_full<<<blocks_for(M.n_copy, 256), 256, 0, st>>>(M, w, xfull);
}

void launch_slots_diff(const DevMesh& M, const double* v, const double* t, double* cbuf, cudaStream_t st) {
  if (M.n_copy > 0) k_slots_diff<<<blocks_for(M.n_copy, 256), 256, 0, st>>>(M, v, t, cbuf);
}

void launch_lumped32(const DevMesh& M, const double* w, const float* kbb32, const long long* kbb_off, double* cbuf,
                     cudaStream_t st, int max_copy) {
  const size_t smem = sizeof(float) * (size_t)(max_copy > 0 ? max_copy : 1);
  static const int lim = dyn_smem_limit((const void*)k_lumped<float>);
  cudaFuncSetAttribute(k_lumped<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  k_lumped<float><<<M.n_sub, 256, smem, st>>>(M, w, kbb32, kbb_off, cbuf);
}

void launch_dot(const double* x, const double* y, long long n, double* partial, double* out, cudaStream_t st) {
  k_dot_partial<<<kRedBlocks, 256, 0, st>>>(x, y, n, partial);
  k_dot_final<<<1, 256, 0, st>>>(partial, kRedBlocks, out);
}

void launch_axpby(long long n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st) {
  if (n > 0) k_axpby<<<blocks_for(n, 256), 256, 0, st>>>(n, a, x, b, y, out);
}

void launch_p_update(long long n, const double* y, double* p, const double* sc, int first, cudaStream_t st) {
  if (n > 0) k_p_update<<<blocks_for(n, 256), 256, 0, st>>>(n, y, p, sc, first);
}

void launch_lam_r_update(long long n, const double* p, const double* Fp, double* lam, double* r, double* sc,
                         cudaStream_t st) {
  k_scalars_after_pfp<<<1, 32, 0, st>>>(sc);
  if (n > 0) k_lam_r_update<<<blocks_for(n, 256), 256, 0, st>>>(n, p, Fp, lam, r, sc);
}

void launch_pcg_init(double* sc, double tol2, int maxit, cudaStream_t st) {
  k_pcg_init<<<1, 32, 0, st>>>(sc, tol2, maxit);
}

void launch_dot2(const double* x1, const double* y1, const double* x2, const double* y2, long long n,
                 double* partial, double* out1, double* out2, cudaStream_t st) {
  k_dot2_partial<<<kRedBlocks, 256, 0, st>>>(x1, y1, x2, y2, n, partial);
  k_dot2_final<<<1, 256, 0, st>>>(partial, kRedBlocks, out1, out2);
}

void launch_GT32_dot(const DevMesh& M, const double* x, const float* h8, double* out, const double* v, int mode,
                     double* sc, double* partial, int* ctr, cudaStream_t st, const double* AW, const double* Einv) {
  if (AW) k_GT32_dot<true><<<kFusedBlocks, 256, 0, st>>>(M, M.GTv32, x, h8, out, v, mode, sc, partial, ctr, AW, Einv);
  else k_GT32_dot<false><<<kFusedBlocks, 256, 0, st>>>(M, M.GTv32, x, h8, out, v, mode, sc, partial, ctr, AW, Einv);
}

void launch_G32_coarse32(const DevMesh& M, const CoarseOp& C, const double* x, double* gx, float* gx32, double* hx,
                         float* hx8, cudaStream_t st) {
  k_G_csr<float><<<M.n_sub, 256, 0, st>>>(M, M.Gv32, x, gx, 1.0, gx32);
  coarse_apply32(C, gx, gx32, hx, hx8, st);
}

void launch_contract_dot(const DevMesh& M, const double* cbuf, double* Fp, const double* p, double* sc,
                         double* partial, int* ctr, cudaStream_t st) {
  k_contract_dot<<<kFusedBlocks, 256, 0, st>>>(M, cbuf, Fp, p, sc, partial, ctr);
}

void launch_lam_r_update_post(long long n, const double* p, const double* Fp, double* lam, double* r, double* sc,
                              int* ctr, unsigned long long h, int has_h, cudaStream_t st) {
  k_lam_r_update_post<<<kFusedBlocks, 256, 0, st>>>(n, p, Fp, lam, r, sc, ctr, (cudaGraphConditionalHandle)h, has_h);
}

void launch_pcg_pre(double* sc, cudaStream_t st) { k_pcg_pre<<<1, 32, 0, st>>>(sc); }
void launch_pcg_mid(double* sc, cudaStream_t st) { k_pcg_mid<<<1, 32, 0, st>>>(sc); }
void launch_pcg_post(double* sc, unsigned long long h, cudaStream_t st) {
  k_pcg_post<<<1, 32, 0, st>>>(sc, (cudaGraphConditionalHandle)h);
}

void launch_p_update_g(long long n, const double* y, double* p, const double* sc, cudaStream_t st, const double* W) {
  if (n > 0) k_p_update_g<<<blocks_for(n, 256), 256, 0, st>>>(n, y, p, sc, W);
}

void launch_lam_r_update_g(long long n, const double* p, const double* Fp, double* lam, double* r, const double* sc,
                           cudaStream_t st) {
  if (n > 0) k_lam_r_update_g<<<blocks_for(n, 256), 256, 0, st>>>(n, p, Fp, lam, r, sc);
}

void launch_coarse_assemble(const DevMesh& M, const int* pair_p, const int* pair_q, const long long* pair_start,
                            const int* trip_group, const int* trip_i, const int* trip_j, long long n_pairs,
                            double* A, long long l, cudaStream_t st) {
  cudaMemsetAsync(A, 0, sizeof(double) * l * l, st);
  if (n_pairs > 0)
    k_coarse_assemble<<<(unsigned)n_pairs, 64, 0, st>>>(M, pair_p, pair_q, pair_start, trip_group, trip_i, trip_j,
                                                         n_pairs, A, l);
}

// In place: A (l x l, symmetric positive definite) -> H = A^{-1}.
// work needs dense_inverse_work(l) doubles.  Blocked Cholesky A = L L^T with
// the inverse of every diagonal block kept, then Y = L^{-1} by block forward
// substitution and H = Y^T Y.  A non-positive pivot sets *err (device).
long long dense_inverse_work(long long l) {
  const long long nblk = (l + kD - 1) / kD;
  return l * l + nblk * kD * kD + kD * l;
}

int dense_cholesky_inverse(double* A, double* work, long long l, int* err, cudaStream_t st) {
  const long long nblk = (l + kD - 1) / kD;
  double* Y = work;                        // l x l
  double* Dall = work + l * l;             // nblk x kD x kD
  double* T = Dall + nblk * kD * kD;       // kD x l
  for (long long b = 0; b < nblk; ++b) {
    const long long k0 = b * kD;
    const int jb = (int)((l - k0) < kD ? (l - k0) : kD);
    double* Dinv = Dall + b * kD * kD;
    k_dense_diag<<<1, 32, 0, st>>>(A, l, k0, jb, Dinv, err);
    const long long rest = l - k0 - jb;
    if (rest > 0) {
      k_dense_panel<<<blocks_for(rest, 8), 256, 0, st>>>(A, l, k0, jb, Dinv);
      dgemm(rest, rest, 0, jb, -1.0, A + (k0 + jb) * l + k0, l, 1, A + (k0 + jb) * l + k0, 1, l, 1.0,
            A + (k0 + jb) * l + (k0 + jb), l, 1, 0, st);
    }
  }
  cudaMemsetAsync(Y, 0, sizeof(double) * l * l, st);
  for (long long b = 0; b < nblk; ++b) {
    const long long k0 = b * kD;
    const int jb = (int)((l - k0) < kD ? (l - k0) : kD);
    const double* Dinv = Dall + b * kD * kD;
    if (k0 > 0) {
      // T = -L[b, 0:k0] Y[0:k0, 0:k0];  Y[b, 0:k0] = Dinv_b T
      dgemm(jb, k0, 0, k0, -1.0, A + k0 * l, l, 1, Y, l, 1, 0.0, T, l, 0, 0, st);
      dgemm(jb, k0, 0, jb, 1.0, Dinv, kD, 1, T, l, 1, 0.0, Y + k0 * l, l, 0, 0, st);
    }
    // Y[b, k0:k0+jb] = Dinv_b (lower triangle; upper part of Dinv is zero)
    cudaMemcpy2DAsync(Y + k0 * l + k0, sizeof(double) * l, Dinv, sizeof(double) * kD, sizeof(double) * jb, jb,
                      cudaMemcpyDeviceToDevice, st);
  }
  // H = Y^T Y
  dgemm(l, l, 0, l, 1.0, Y, 1, l, Y, l, 1, 0.0, A, l, 0, 1, st);
  return 0;
}


void launch_coarse_assemble_planes(const DevMesh& M, const int* pair_p, const int* pair_q, const long long* pair_start,
                                   const int* trip_group, const int* trip_i, const int* trip_j, long long n_pairs,
                                   double* Adiag, double* Aoff, int per_plane, int n_pl, int n_planes,
                                   cudaStream_t st) {
  const size_t blk = (size_t)n_pl * n_pl;
  cudaMemsetAsync(Adiag, 0, sizeof(double) * blk * n_planes, st);
  cudaMemsetAsync(Aoff, 0, sizeof(double) * blk * n_planes, st);
  if (n_pairs > 0)
    k_coarse_assemble_planes<<<(unsigned)n_pairs, 64, 0, st>>>(M, pair_p, pair_q, pair_start, trip_group, trip_i,
                                                                trip_j, n_pairs, Adiag, Aoff, per_plane, n_pl);
}

// Block LDL^T of the block-tridiagonal G G^T over the planes, with explicit inverses:
// D_0 = A_00, D_k = A_kk - A_{k,k-1} W_{k-1} A_{k,k-1}^T, W_k = D_k^-1 (in place of Adiag),
// V_k = W_k A_{k,k-1} (k >= 1), U_k = W_k A_{k+1,k}^T (k <= np-2).  T: n_pl^2 doubles,
// work: dense_inverse_work(n_pl) doubles.  A non-positive pivot sets *err (device).
void coarse_planes_factor(double* W, const double* Aoff, double* V, double* U, int n, int np, double* T,
                          double* work, int* err, cudaStream_t st) {
  const long long blk = (long long)n * n;
  for (int k = 0; k < np; ++k) {
    double* Wk = W + k * blk;
    if (k > 0) {
      const double* Ak = Aoff + k * blk;
      dgemm(n, n, 0, n, 1.0, Ak, n, 1, W + (k - 1) * blk, n, 1, 0.0, T, n, 0, 0, st);   // T = A_{k,k-1} W_{k-1}
      dgemm(n, n, 0, n, -1.0, T, n, 1, Ak, 1, n, 1.0, Wk, n, 0, 0, st);                // D_k = A_kk - T A^T
    }
    dense_cholesky_inverse(Wk, work, n, err, st);
  }
  for (int k = 0; k < np; ++k) {
    const double* Wk = W + k * blk;
    if (k > 0) dgemm(n, n, 0, n, 1.0, Wk, n, 1, Aoff + k * blk, n, 1, 0.0, V + k * blk, n, 0, 0, st);
    if (k + 1 < np) dgemm(n, n, 0, n, 1.0, Wk, n, 1, Aoff + (k + 1) * blk, 1, n, 0.0, U + k * blk, n, 0, 0, st);
  }
}

template <typename T>
static void plane_apply(const T* W, const T* V, const T* U, int n, int np, const double* x, double alpha, double* y,
                        float* y8, cudaStream_t st) {
  const unsigned rb = (unsigned)((n + kPlaneRows - 1) / kPlaneRows);
  const size_t smem = sizeof(T) * (size_t)n;
  const long long blk = (long long)n * n;
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_plane_first<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_plane_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  k_plane_first<T><<<dim3(rb, (unsigned)np), 256, smem, st>>>(W, n, x, alpha, y, y8, np == 1 ? 1 : 0);
  for (int k = 1; k < np; ++k)
    k_plane_step<T><<<rb, 256, smem, st>>>(V + k * blk, n, y + (long long)(k - 1) * n, y + (long long)k * n,
                                           (long long)k * n, y8, k == np - 1 ? 1 : 0);
  for (int k = np - 2; k >= 0; --k)
    k_plane_step<T><<<rb, 256, smem, st>>>(U + k * blk, n, y + (long long)(k + 1) * n, y + (long long)k * n,
                                           (long long)k * n, y8, 1);
}

void coarse_apply(const CoarseOp& C, const double* x, double alpha, double* y, cudaStream_t st) {
  if (C.mode == kCoarseDense) {
    launch_gemv(C.H, C.l, x, alpha, y, st);
  } else {
    plane_apply<double>(C.W, C.V, C.U, C.n_pl, C.n_planes, x, alpha, y, nullptr, st);
  }
}

void coarse_apply32(const CoarseOp& C, const double* x, const float* x32, double* y, float* y8, cudaStream_t st) {
  if (C.mode == kCoarseDense) {
    static const int lim = dyn_smem_limit((const void*)k_gemv32);
    cudaFuncSetAttribute(k_gemv32, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    const long long ld = h32_ld(C.l);
    k_gemv32<<<blocks_for(C.l, kGemvRows), 512, sizeof(float) * (size_t)ld, st>>>(C.H32, C.l, ld, x, x32, y, y8);
  } else {
    plane_apply<float>(C.W32, C.V32, C.U32, C.n_pl, C.n_planes, x, 1.0, y, y8, st);
  }
}

int coarse_launches(const CoarseOp& C) { return C.mode == kCoarseDense ? 1 : 2 * C.n_planes - 1; }

}  // namespace tfeti
