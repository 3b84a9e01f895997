// Subdomains with few plastic Gauss points on their shape's elastic factor plus a low-rank
// correction (Sherman-Morrison-Woodbury), instead of a refactorisation.
//
// The assembled tangent of a subdomain with plastic Gauss points differs from its shape's
// elastic matrix by the element corrections of Algorithm 5's Clarke tangent (Sec. 3.1):
//   K_p = K_el - sum_{plastic g} |T| B_g^T (a_g E_eps + b_g n_g n_g^T) B_g = K_el - U U^T,
// with six columns per plastic point, U_g = sqrt(a_g |T|) B_g^T F and sqrt(b_g |T|) B_g^T n_g,
// F F^T = E_eps (F: an orthonormal basis of the deviatoric plane, and sqrt(1/2) on the shear
// components).  a_g, b_g >= 0 and the tangent stays positive definite, so with the fixing-dof
// generalised inverse K^+ of the elastic matrix (zero rows and columns at the fixing dofs of
// Remark 1), the fixing-dof generalised inverse of K_p is
//   K_p^+ = K^+ + Z C^{-1} Z^T,  Z = K^+ U,  C = I - U^T K^+ U = I - U^T Z,
// C symmetric positive definite (K_p restricted to the free dofs is).
//
// Set-up, once per assembly, in FP64 from the shape's dense FP64 K^+ (all subdomains of the list
// in each launch): the plastic points in order (k_wood_points), U and the points' dofs (k_wood_U),
// Z^T over all n dofs (k_wood_Z), C (k_wood_C), its blocked Cholesky factor L (k_wood_chol_*).
// From these, for the FP32 inner F-apply: L rounded to FP32, Z_b^T (the boundary columns of Z^T)
// in FP32 and Y = C^{-1} Z_b^T by blocked FP32 substitution (k_wood_subst), so that on the box
// boundary S_p = S_el + Z_b Y: the subdomain's slots come from the shape's tensor-core GEMM (as
// for elastic subdomains) plus Z_b (Y x_b) (k_wood_t with the gather of x_b, then k_wood_y).
//
// FP64 subdomain solves (residual solves, F-applies, K^+ applies) of these subdomains run on the
// shape's elastic factor and the correction Z C^{-1} Z^T v is added after them: k_wood_v64 forms
// the solve's right-hand side v, k_wood_t64 t = Z^T v, k_wood_s64 s = C^{-1} t by blocked forward
// and backward substitution with L, k_wood_y64 y = Z s on all dofs, k_wood_cb64 y at the copy
// slots.
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

// element node offsets (same order as the shape-function gradient table dN)
__constant__ int c_wnode[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                  {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

// columns of F (Voigt order xx, yy, zz, xy, yz, xz): deviatoric plane basis, then sqrt(1/2) on
// each shear component
__constant__ double c_wF[5][6] = {{0.70710678118654752440, -0.70710678118654752440, 0, 0, 0, 0},
                                  {0.40824829046386301637, 0.40824829046386301637, -0.81649658092772603273, 0, 0, 0},
                                  {0, 0, 0, 0.70710678118654752440, 0, 0},
                                  {0, 0, 0, 0, 0.70710678118654752440, 0},
                                  {0, 0, 0, 0, 0, 0.70710678118654752440}};

// Plastic points of subdomain list[w] in Gauss-point order -> pts + pt_off[w] (a block-wide scan).
__global__ void k_wood_points(DevMesh M, const int* __restrict__ list, const long long* __restrict__ pt_off,
                              const int* __restrict__ n_pts, const uint8_t* __restrict__ plastic, int* pts) {
  __shared__ int wsum[32];
  __shared__ int base;
  const SubDev S = M.subs[list[blockIdx.x]];
  const long long g0 = 8 * S.elem_off;
  const int n = 8 * S.n_elem;
  int* out = pts + pt_off[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c = 0; c < n; c += blockDim.x) {
    const int i = c + threadIdx.x;
    const bool f = i < n && plastic[g0 + i] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = base;
    for (int k = 0; k < warp; ++k) before += wsum[k];
    const int at = before + __popc(bal & ((1u << lane) - 1u));
    if (f && at < n_pts[blockIdx.x]) out[at] = i;   // the count equals n_pts (same flags)
    __syncthreads();
    if (threadIdx.x == 0)
      for (int k = 0; k < nw; ++k) base += wsum[k];
    __syncthreads();
  }
}

// U and the local dofs of point i = blockIdx.y of subdomain list[blockIdx.x]: lane t < 24 takes
// element dof t (node t / 3, component t % 3).  U row 6i + j at u_pool + 144 (pt_off + i) + 24 j.
__global__ void k_wood_U(DevMesh M, WoodArgs a) {
  const int w = blockIdx.x, i = blockIdx.y, t = threadIdx.x;
  if (i >= a.n_pts[w] || t >= 24) return;
  const SubDev S = M.subs[a.list[w]];
  const long long po = a.pt_off[w] + i;
  const int pt = a.pts[po];
  const int le = pt >> 3, g = pt & 7;
  const int ax = S.dims[0], ay = S.dims[1];
  const int ex = le % ax, ey = (le / ax) % ay, ez = le / (ax * ay);
  const long long gp = 8 * (S.elem_off + le) + g;
  const double sa = sqrt(fmax(a.pa[gp], 0.0) * M.wdet), sb = sqrt(fmax(a.pb[gp], 0.0) * M.wdet);
  const int nd = t / 3, comp = t % 3;
  const int ln = (ex + c_wnode[nd][0]) + S.nn[0] * ((ey + c_wnode[nd][1]) + S.nn[1] * (ez + c_wnode[nd][2]));
  a.dof_pool[24 * po + t] = 3 * ln + comp;
  const double dx = M.dN[(g * 8 + nd) * 3], dy = M.dN[(g * 8 + nd) * 3 + 1], dz = M.dN[(g * 8 + nd) * 3 + 2];
  for (int j = 0; j < 6; ++j) {
    double v[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = j < 5 ? c_wF[j][q] : a.pn[q * M.n_gp + gp];
    const double s = j < 5 ? sa : sb;
    double u;
    if (comp == 0) u = dx * v[0] + dy * v[3] + dz * v[5];
    else if (comp == 1) u = dy * v[1] + dx * v[3] + dz * v[4];
    else u = dz * v[2] + dy * v[4] + dx * v[5];
    a.u_pool[144 * po + 24 * j + t] = s * u;
  }
}

// Z^T rows 6i..6i+5 (i = blockIdx.y) of subdomain list[blockIdx.x] over all its n dofs:
// Zt[6i + q][k] = sum_t U[6i + q][t] K^+[D_i[t]][k]  (K^+ symmetric: rows D_i[t] are contiguous).
__global__ void __launch_bounds__(256) k_wood_Z(DevMesh M, WoodArgs a) {
  __shared__ int di[24];
  __shared__ double ui[6][24];
  const int w = blockIdx.x, i = blockIdx.y;
  if (i >= a.n_pts[w]) return;
  const SubDev S = M.subs[a.list[w]];
  const int n = S.n_dof;
  const double* K = a.kinv + a.kinv_off[S.shape];
  const long long po = a.pt_off[w] + i;
  for (int e = threadIdx.x; e < 144; e += blockDim.x) ui[e / 24][e % 24] = a.u_pool[144 * po + e];
  if (threadIdx.x < 24) di[threadIdx.x] = a.dof_pool[24 * po + threadIdx.x];
  __syncthreads();
  double* Zt = a.zt_pool + a.zt_off[w] + (long long)(6 * i) * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int t = 0; t < 24; ++t) {
      const double kv = __ldg(K + (long long)di[t] * n + k);
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] = fma(ui[q][t], kv, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) Zt[(long long)q * n + k] = acc[q];
  }
}

// C rows 6i..6i+5 (i = blockIdx.y) of subdomain list[blockIdx.x]: C[6i + q][c] = delta -
// sum_t U[6i + q][t] Zt[c][D_i[t]], one warp per column c (lane t < 24 takes dof t).
__global__ void __launch_bounds__(256) k_wood_C(DevMesh M, WoodArgs a) {
  const int w = blockIdx.x, i = blockIdx.y;
  const int np = a.n_pts[w];
  if (i >= np) return;
  const SubDev S = M.subs[a.list[w]];
  const int n = S.n_dof, r = 6 * np;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long po = a.pt_off[w] + i;
  double u[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int d = 0;
  if (lane < 24) {
    d = a.dof_pool[24 * po + lane];
#pragma unroll
    for (int q = 0; q < 6; ++q) u[q] = a.u_pool[144 * po + 24 * q + lane];
  }
  const double* Zt = a.zt_pool + a.zt_off[w];
  double* C = a.c_pool + a.c_off[w];
  for (int c = warp; c < r; c += blockDim.x >> 5) {
    const double z = lane < 24 ? Zt[(long long)c * n + d] : 0.0;
    double p[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      p[q] = u[q] * z;
      for (int o = 16; o > 0; o >>= 1) p[q] += __shfl_xor_sync(0xffffffffu, p[q], o);
    }
    if (lane < 6) {
      double v = p[0];
#pragma unroll
      for (int q = 1; q < 6; ++q) v = lane == q ? p[q] : v;
      C[(long long)(6 * i + lane) * r + c] = (6 * i + lane == c ? 1.0 : 0.0) - v;
    }
  }
}

// Blocked Cholesky C = L L^T in place (lower triangle), panels of kBlk columns, all subdomains
// in each launch: for panel p, k_wood_chol_diag factors the diagonal block (one CTA per
// subdomain, in shared memory) and stores the inverse of its factor in d_pool (kBlk x kBlk per
// panel); k_wood_chol_trsm forms the panel below it, L_ip = C_ip L_pp^-T; k_wood_chol_syrk
// updates the trailing lower triangle, C_ij -= L_ip L_jp^T, one kBlk x kBlk tile per CTA.
// A non-positive pivot sets *err bit 8 (the host then refactorises these subdomains).
constexpr int kBlk = 32;

__device__ __forceinline__ int wood_nblk(int r) { return (r + kBlk - 1) / kBlk; }

__global__ void __launch_bounds__(256) k_wood_chol_diag(WoodArgs a, int p) {
  __shared__ double A[kBlk][kBlk + 1], Li[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * a.n_pts[w];
  const int k0 = p * kBlk;
  if (k0 >= r) return;
  const int jb = min(kBlk, r - k0);
  double* C = a.c_pool + a.c_off[w];
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    A[i][j] = (i < jb && j < jb) ? C[(long long)(k0 + i) * r + k0 + j] : (i == j ? 1.0 : 0.0);
    Li[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < kBlk; ++k) {   // right-looking in shared memory
    if (threadIdx.x == 0) {
      if (!(A[k][k] > 0.0)) atomicOr(a.err, 8);
      A[k][k] = sqrt(fmax(A[k][k], 1e-300));
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < kBlk; i += blockDim.x) A[i][k] /= A[k][k];
    __syncthreads();
    for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
      const int i = e / kBlk, j = e % kBlk;
      if (i > k && j > k && j <= i) A[i][j] -= A[i][k] * A[j][k];
    }
    __syncthreads();
  }
  // inverse of the lower factor, one column per thread (forward substitution of unit vectors)
  if (threadIdx.x < kBlk) {
    const int c = threadIdx.x;
    for (int i = 0; i < kBlk; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int q = c; q < i; ++q) v -= A[i][q] * Li[q][c];
      Li[i][c] = i >= c ? v / A[i][i] : 0.0;
    }
  }
  __syncthreads();
  double* D = a.d_pool + a.d_off[w] + (long long)p * kBlk * kBlk;
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    D[e] = Li[i][j];
    if (i < jb && j < jb && j <= i) C[(long long)(k0 + i) * r + k0 + j] = A[i][j];
  }
}

__global__ void __launch_bounds__(256) k_wood_chol_trsm(WoodArgs a, int p) {
  __shared__ double X[kBlk][kBlk + 1], Li[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * a.n_pts[w];
  const int k0 = p * kBlk, i0 = (p + 1 + blockIdx.y) * kBlk;
  if (i0 >= r) return;
  const int ib = min(kBlk, r - i0), jb = min(kBlk, r - k0);
  double* C = a.c_pool + a.c_off[w];
  const double* D = a.d_pool + a.d_off[w] + (long long)p * kBlk * kBlk;
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    X[i][j] = (i < ib && j < jb) ? C[(long long)(i0 + i) * r + k0 + j] : 0.0;
    Li[i][j] = D[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {   // L_ip = X Li^T
    const int i = e / kBlk, j = e % kBlk;
    if (i >= ib || j >= jb) continue;
    double v = 0.0;
    for (int q = 0; q <= j; ++q) v += X[i][q] * Li[j][q];
    C[(long long)(i0 + i) * r + k0 + j] = v;
  }
}

__global__ void __launch_bounds__(256) k_wood_chol_syrk(WoodArgs a, int p) {
  __shared__ double Li[kBlk][kBlk + 1], Lj[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * a.n_pts[w];
  const int nb = wood_nblk(r) - p - 1;            // trailing blocks
  // tile t of the trailing lower triangle: (bi, bj), bj <= bi
  int t = blockIdx.y, bi = 0;
  while (bi < nb && t > bi) t -= ++bi;
  if (bi >= nb) return;
  const int bj = t;
  const int k0 = p * kBlk, i0 = (p + 1 + bi) * kBlk, j0 = (p + 1 + bj) * kBlk;
  const int ib = min(kBlk, r - i0), jb = min(kBlk, r - j0), kb = min(kBlk, r - k0);
  double* C = a.c_pool + a.c_off[w];
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, q = e % kBlk;
    Li[i][q] = (i < ib && q < kb) ? C[(long long)(i0 + i) * r + k0 + q] : 0.0;
    Lj[i][q] = (i < jb && q < kb) ? C[(long long)(j0 + i) * r + k0 + q] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    if (i >= ib || j >= jb || (bi == bj && j > i)) continue;
    double v = 0.0;
#pragma unroll 8
    for (int q = 0; q < kBlk; ++q) v += Li[i][q] * Lj[j][q];
    C[(long long)(i0 + i) * r + j0 + j] -= v;
  }
}

// Z_b^T in FP32: row c (one warp each, blockIdx.y * 8 + warp) of subdomain list[blockIdx.x],
// zb[c][k] = Zt[c][boundary dof k].
__global__ void __launch_bounds__(256) k_wood_Zb32(DevMesh M, WoodArgs a) {
  const int w = blockIdx.x;
  const int r = 6 * a.n_pts[w];
  const int lane = threadIdx.x & 31, c = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (c >= r) return;
  const SubDev S = M.subs[a.list[w]];
  const int n = S.n_dof, n_bd = 3 * S.n_bnd;
  const double* zr = a.zt_pool + a.zt_off[w] + (long long)c * n;
  float* out = a.z_pool + a.z_off[w] + (long long)c * n_bd;
  for (int k = lane; k < n_bd; k += 32) out[k] = (float)zr[3 * M.shape_bln[S.bnd_off + k / 3] + k % 3];
}

// Y = C^-1 Z_b^T in place of the r x n_bd array Y (a copy of Z_b^T), FP32, for 32 boundary
// columns per CTA (blockIdx.y): forward Y_b = Li_b (Y_b - sum_{a<b} L_ba Y_a), then backward
// Y_b = Li_b^T (Y_b - sum_{a>b} L_ab^T Y_a), with L and the inverses Li_b of its diagonal blocks
// rounded to FP32.  The column chunk of Y sits in shared memory (r x 32 floats).
__global__ void __launch_bounds__(256) k_wood_subst(const SubDev* __restrict__ subs, WoodArgs a) {
  extern __shared__ float ys[];     // [r][kBlk]
  __shared__ float T[kBlk][kBlk + 1];
  const int w = blockIdx.x, r = 6 * a.n_pts[w];
  const int n_bd = 3 * subs[a.list[w]].n_bnd;
  const int col0 = blockIdx.y * kBlk;
  if (col0 >= n_bd) return;
  const int cb = min(kBlk, n_bd - col0);
  const float* C = a.c32_pool + a.c_off[w];
  const float* D = a.d32_pool + a.d_off[w];
  float* Y = a.y_pool + a.z_off[w];
  for (int e = threadIdx.x; e < r * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    ys[e] = j < cb ? Y[(long long)i * n_bd + col0 + j] : 0.f;
  }
  __syncthreads();
  const int nbk = wood_nblk(r);
  for (int pass = 0; pass < 2; ++pass) {
    for (int s = 0; s < nbk; ++s) {
      const int b = pass == 0 ? s : nbk - 1 - s;
      const int b0 = b * kBlk, bb = min(kBlk, r - b0);
      // T = Y_b - sum over the solved blocks (forward: a < b, L_ba; backward: a > b, L_ab^T)
      for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
        const int i = e / kBlk, j = e % kBlk;
        float v = i < bb ? ys[(b0 + i) * kBlk + j] : 0.f;
        if (i < bb) {
          if (pass == 0) {
            for (int q = 0; q < b0; ++q) v -= C[(long long)(b0 + i) * r + q] * ys[q * kBlk + j];
          } else {
            for (int q = b0 + bb; q < r; ++q) v -= C[(long long)q * r + b0 + i] * ys[q * kBlk + j];
          }
        }
        T[i][j] = v;
      }
      __syncthreads();
      const float* Li = D + (long long)b * kBlk * kBlk;
      for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
        const int i = e / kBlk, j = e % kBlk;
        if (i >= bb) continue;
        float v = 0.f;
        if (pass == 0)
          for (int q = 0; q <= i; ++q) v += Li[i * kBlk + q] * T[q][j];
        else
          for (int q = i; q < bb; ++q) v += Li[q * kBlk + i] * T[q][j];
        ys[(b0 + i) * kBlk + j] = v;
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < r * kBlk; e += blockDim.x) {
    const int i = e / kBlk, j = e % kBlk;
    if (j < cb) Y[(long long)i * n_bd + col0 + j] = ys[e];
  }
}

// Correction of the inner F-apply, in three launches spread over many CTAs (the per-subdomain
// products are a few MB each and one CTA per subdomain would leave them latency-bound):
// k_wood_t: t = Y x_b for the rows kWoodRows blockIdx.y .. + kWoodRows - 1 of subdomain list[blockIdx.x],
// one row per warp, -> tbuf + w * tstride; each CTA with rows first gathers x_b = B^T lam at the
// subdomain's boundary dofs into shared memory (kXU dofs per thread with their loads in flight).
// k_wood_y: cbuf[slots] += Z_b t for 64 boundary dofs per CTA (blockIdx.y), four threads per dof
// splitting the sum over the rows, combined in shared memory in a fixed order.
constexpr int kWoodRows = 8;
constexpr int kXU = 4;

__global__ void __launch_bounds__(256) k_wood_t(DevMesh M, const int* __restrict__ list, const double* __restrict__ lam,
                                                const int* __restrict__ n_pts, const long long* __restrict__ y_off,
                                                const float* __restrict__ y_pool, float* tbuf, int tstride) {
  extern __shared__ __align__(16) float xb[];
  const int w = blockIdx.x;
  const int r = 6 * n_pts[w];
  if ((int)blockIdx.y * kWoodRows >= r) return;   // the same for the whole CTA
  const SubDev S = M.subs[list[w]];
  const int n_bd = 3 * S.n_bnd;
  for (int k0 = threadIdx.x; k0 < n_bd; k0 += kXU * blockDim.x) {
    long long slot[kXU];
    double v[kXU];
#pragma unroll
    for (int u = 0; u < kXU; ++u) {
      const int k = k0 + u * (int)blockDim.x;
      const int sl = k < n_bd ? __ldg(M.sub_b2s + S.b2s_off + k / 3) : -1;
      slot[u] = sl >= 0 ? (long long)sl + k % 3 : -1;
    }
    bt_at_slots<kXU>(M, lam, slot, v);
#pragma unroll
    for (int u = 0; u < kXU; ++u) {
      const int k = k0 + u * (int)blockDim.x;
      if (k < n_bd) xb[k] = (float)v[u];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * kWoodRows + warp;
  if (c >= r) return;
  const float* yr = y_pool + y_off[w] + (long long)c * n_bd;
  float v = 0.f;
#pragma unroll 8
  for (int k = lane; k < n_bd; k += 32) v += __ldg(yr + k) * xb[k];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) tbuf[(long long)w * tstride + c] = v;
}

__global__ void __launch_bounds__(256) k_wood_y(DevMesh M, const int* __restrict__ list, const int* __restrict__ n_pts,
                                                const long long* __restrict__ z_off, const float* __restrict__ z_pool,
                                                const float* __restrict__ tbuf, int tstride, double* cbuf) {
  __shared__ float part[4][64];
  const int w = blockIdx.x;
  const int r = 6 * n_pts[w];
  const SubDev S = M.subs[list[w]];
  const int n_bd = 3 * S.n_bnd;
  const int k0 = blockIdx.y * 64;
  if (k0 >= n_bd) return;
  const int kk = threadIdx.x & 63, q = threadIdx.x >> 6, k = k0 + kk;
  const float* Zt = z_pool + z_off[w];
  const float* t = tbuf + (long long)w * tstride;
  float v = 0.f;
  if (k < n_bd) {
    const int c0 = q * ((r + 3) / 4), c1 = min(r, c0 + (r + 3) / 4);
#pragma unroll 4
    for (int c = c0; c < c1; ++c) v += __ldg(Zt + (long long)c * n_bd + k) * __ldg(t + c);
  }
  part[q][kk] = v;
  __syncthreads();
  if (q == 0 && k < n_bd) {
    const int sl = M.sub_b2s[S.b2s_off + k / 3];
    if (sl >= 0) cbuf[(long long)sl + k % 3] += (double)(((part[0][kk] + part[1][kk]) + part[2][kk]) + part[3][kk]);
  }
}

// ---- FP64 correction after the subdomain solves with the elastic factor ----------------------
// k_wood_v64: the solve's right-hand side of subdomain list[blockIdx.x], v = src (or 0) +
// sign * B^T lam at its copy slots (each slot has its own local dof), -> vbuf + w * max_n.
__global__ void __launch_bounds__(256) k_wood_v64(DevMesh M, WoodArgs a, const double* __restrict__ src,
                                                  const double* __restrict__ lam, double sign) {
  const int w = blockIdx.x;
  const SubDev S = M.subs[a.list[w]];
  double* v = a.vbuf + (long long)w * a.max_n;
  for (int i = threadIdx.x; i < S.n_dof; i += blockDim.x) v[i] = src ? src[S.dof_off + i] : 0.0;
  __syncthreads();
  if (!lam) return;
  for (int s = threadIdx.x; s < S.n_copy; s += blockDim.x) {
    const long long slot = S.copy_off + s;
    v[M.slot_ldof[slot]] += sign * bt_at_slot(M, lam, slot);
  }
}

// k_wood_t64: t = Z^T v, one row per warp, kWoodRows rows per CTA -> tbuf64 + w * 6 max_pts.
__global__ void __launch_bounds__(256) k_wood_t64(const SubDev* __restrict__ subs, WoodArgs a) {
  const int w = blockIdx.x;
  const int r = 6 * a.n_pts[w];
  const int lane = threadIdx.x & 31, c = blockIdx.y * kWoodRows + (threadIdx.x >> 5);
  if (c >= r) return;
  const int n = subs[a.list[w]].n_dof;
  const double* zr = a.zt_pool + a.zt_off[w] + (long long)c * n;
  const double* v = a.vbuf + (long long)w * a.max_n;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s = fma(__ldg(zr + k), v[k], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) a.tbuf64[(long long)w * 6 * a.max_pts + c] = s;
}

// k_wood_s64: t <- C^-1 t in place for subdomain list[blockIdx.x] (one CTA, 256 threads):
// forward s_b = Li_b (t_b - L_{b,<b} s_{<b}), one warp per row of the block; then backward
// s_b = Li_b^T (s_b - L_{>b,b}^T s_{>b}), the column sums split over the eight warps and added in
// warp order.
__global__ void __launch_bounds__(256) k_wood_s64(WoodArgs a) {
  __shared__ double s[6 * kWoodMaxPts];
  __shared__ double T[kBlk];
  __shared__ double part[8][kBlk];
  const int w = blockIdx.x, r = 6 * a.n_pts[w];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* L = a.c_pool + a.c_off[w];
  const double* D = a.d_pool + a.d_off[w];
  double* t = a.tbuf64 + (long long)w * 6 * a.max_pts;
  for (int c = tid; c < r; c += blockDim.x) s[c] = t[c];
  __syncthreads();
  const int nbk = wood_nblk(r);
  for (int b = 0; b < nbk; ++b) {
    const int b0 = b * kBlk, bb = min(kBlk, r - b0);
    for (int i = warp; i < bb; i += 8) {
      const double* row = L + (long long)(b0 + i) * r;
      double v = 0.0;
      for (int q = lane; q < b0; q += 32) v = fma(row[q], s[q], v);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) T[i] = s[b0 + i] - v;
    }
    __syncthreads();
    if (tid < bb) {
      const double* Li = D + (long long)b * kBlk * kBlk + tid * kBlk;
      double v = 0.0;
      for (int q = 0; q <= tid; ++q) v = fma(Li[q], T[q], v);
      s[b0 + tid] = v;
    }
    __syncthreads();
  }
  for (int b = nbk - 1; b >= 0; --b) {
    const int b0 = b * kBlk, bb = min(kBlk, r - b0);
    double v = 0.0;
    if (lane < bb)
      for (int q = b0 + bb + warp; q < r; q += 8) v = fma(L[(long long)q * r + b0 + lane], s[q], v);
    part[warp][lane] = v;
    __syncthreads();
    if (tid < bb) {
      double acc = 0.0;
      for (int k = 0; k < 8; ++k) acc += part[k][tid];
      T[tid] = s[b0 + tid] - acc;
    }
    __syncthreads();
    if (tid < bb) {
      const double* Li = D + (long long)b * kBlk * kBlk;
      double x = 0.0;
      for (int q = tid; q < bb; ++q) x = fma(Li[q * kBlk + tid], T[q], x);
      s[b0 + tid] = x;
    }
    __syncthreads();
  }
  for (int c = tid; c < r; c += blockDim.x) t[c] = s[c];
}

// k_wood_y64: y = Z s for 64 dofs per CTA (blockIdx.y), four threads per dof splitting the rows,
// combined in a fixed order; dst (the subdomain's part of the decomposed vector) += y where
// given, y -> ybuf + w * max_n.
__global__ void __launch_bounds__(256) k_wood_y64(DevMesh M, WoodArgs a, double* dst) {
  __shared__ double part[4][64];
  const int w = blockIdx.x;
  const int r = 6 * a.n_pts[w];
  const SubDev S = M.subs[a.list[w]];
  const int n = S.n_dof;
  const int k0 = blockIdx.y * 64;
  if (k0 >= n) return;
  const int kk = threadIdx.x & 63, q = threadIdx.x >> 6, k = k0 + kk;
  const double* Zt = a.zt_pool + a.zt_off[w];
  const double* sv = a.tbuf64 + (long long)w * 6 * a.max_pts;
  double v = 0.0;
  if (k < n) {
    const int c0 = q * ((r + 3) / 4), c1 = min(r, c0 + (r + 3) / 4);
    for (int c = c0; c < c1; ++c) v = fma(__ldg(Zt + (long long)c * n + k), sv[c], v);
  }
  part[q][kk] = v;
  __syncthreads();
  if (q == 0 && k < n) {
    const double y = ((part[0][kk] + part[1][kk]) + part[2][kk]) + part[3][kk];
    a.ybuf[(long long)w * a.max_n + k] = y;
    if (dst) dst[S.dof_off + k] += y;
  }
}

// k_wood_cb64: cbuf at the copy slots of subdomain list[blockIdx.x] += y at the slot's local dof.
__global__ void __launch_bounds__(256) k_wood_cb64(DevMesh M, WoodArgs a, double* cbuf) {
  const int w = blockIdx.x;
  const SubDev S = M.subs[a.list[w]];
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= S.n_copy) return;
  const long long slot = S.copy_off + s;
  cbuf[slot] += a.ybuf[(long long)w * a.max_n + M.slot_ldof[slot]];
}

}  // namespace

void launch_wood_setup(const DevMesh& M, const WoodArgs& a, cudaStream_t st) {
  if (a.n <= 0) return;
  const dim3 gp((unsigned)a.n, (unsigned)a.max_pts);
  k_wood_points<<<a.n, 256, 0, st>>>(M, a.list, a.pt_off, a.n_pts, a.plastic, a.pts);
  k_wood_U<<<gp, 32, 0, st>>>(M, a);
  k_wood_Z<<<gp, 256, 0, st>>>(M, a);
  k_wood_C<<<gp, 256, 0, st>>>(M, a);
  const int rmax = 6 * a.max_pts, nb = (rmax + kBlk - 1) / kBlk;
  for (int p = 0; p < nb; ++p) {
    k_wood_chol_diag<<<a.n, 256, 0, st>>>(a, p);
    if (p + 1 < nb) {
      const int t = nb - p - 1;
      k_wood_chol_trsm<<<dim3((unsigned)a.n, (unsigned)t), 256, 0, st>>>(a, p);
      k_wood_chol_syrk<<<dim3((unsigned)a.n, (unsigned)(t * (t + 1) / 2)), 256, 0, st>>>(a, p);
    }
  }
  // the inner (FP32) apply's data: L and the diagonal inverses rounded, Z_b^T, Y = C^-1 Z_b^T
  launch_to_f32(a.c_pool, a.c32_pool, a.c_total, st);
  launch_to_f32(a.d_pool, a.d32_pool, a.d_total, st);
  k_wood_Zb32<<<dim3((unsigned)a.n, (unsigned)((rmax + 7) / 8)), 256, 0, st>>>(M, a);
  cudaMemcpyAsync(a.y_pool, a.z_pool, sizeof(float) * (size_t)a.z_total, cudaMemcpyDeviceToDevice, st);
  const size_t smem = sizeof(float) * (size_t)rmax * kBlk;
  cudaFuncSetAttribute(k_wood_subst, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_wood_subst<<<dim3((unsigned)a.n, (unsigned)((a.max_bd + kBlk - 1) / kBlk)), 256, smem, st>>>(M.subs, a);
}

int wood_setup_launches(const WoodArgs& a) {
  const int nb = (6 * a.max_pts + kBlk - 1) / kBlk;
  return 4 + (3 * nb - 2) + 4;
}

void launch_wood_apply(const DevMesh& M, const WoodArgs& a, const double* lam, double* cbuf, cudaStream_t st) {
  if (a.n <= 0) return;
  const int rmax = 6 * a.max_pts;
  static const int lim = dyn_smem_limit((const void*)k_wood_t);
  cudaFuncSetAttribute(k_wood_t, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  k_wood_t<<<dim3((unsigned)a.n, (unsigned)((rmax + kWoodRows - 1) / kWoodRows)), 256, sizeof(float) * (size_t)a.max_bd,
             st>>>(M, a.list, lam, a.n_pts, a.z_off, a.y_pool, a.tbuf, rmax);
  k_wood_y<<<dim3((unsigned)a.n, (unsigned)((a.max_bd + 63) / 64)), 256, 0, st>>>(M, a.list, a.n_pts, a.z_off,
                                                                                   a.z_pool, a.tbuf, rmax, cbuf);
}

// dst += y at the dofs of subdomain list[blockIdx.x] (y from k_wood_y64 in ybuf).
__global__ void __launch_bounds__(256) k_wood_add64(DevMesh M, WoodArgs a, double* dst) {
  const int w = blockIdx.x;
  const SubDev S = M.subs[a.list[w]];
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= S.n_dof) return;
  dst[S.dof_off + k] += a.ybuf[(long long)w * a.max_n + k];
}

int launch_wood_corr64(const DevMesh& M, const WoodArgs& a, const double* src, const double* lam, double sign,
                       cudaStream_t st) {
  if (a.n <= 0) return 0;
  const int rmax = 6 * a.max_pts;
  k_wood_v64<<<a.n, 256, 0, st>>>(M, a, src, lam, sign);
  k_wood_t64<<<dim3((unsigned)a.n, (unsigned)((rmax + kWoodRows - 1) / kWoodRows)), 256, 0, st>>>(M.subs, a);
  k_wood_s64<<<a.n, 256, 0, st>>>(a);
  k_wood_y64<<<dim3((unsigned)a.n, (unsigned)((a.max_n + 63) / 64)), 256, 0, st>>>(M, a, nullptr);
  return 4;
}

int launch_wood_add64(const DevMesh& M, const WoodArgs& a, double* cbuf, double* dst, cudaStream_t st) {
  if (a.n <= 0) return 0;
  int n = 0;
  if (dst) {
    k_wood_add64<<<dim3((unsigned)a.n, (unsigned)((a.max_n + 255) / 256)), 256, 0, st>>>(M, a, dst);
    ++n;
  }
  if (cbuf) {
    k_wood_cb64<<<dim3((unsigned)a.n, (unsigned)((a.max_copy + 255) / 256)), 256, 0, st>>>(M, a, cbuf);
    ++n;
  }
  return n;
}

int launch_wood_apply64(const DevMesh& M, const WoodArgs& a, const double* src, const double* lam, double sign,
                        double* cbuf, double* dst, cudaStream_t st) {
  if (a.n <= 0) return 0;
  const int rmax = 6 * a.max_pts;
  k_wood_v64<<<a.n, 256, 0, st>>>(M, a, src, lam, sign);
  k_wood_t64<<<dim3((unsigned)a.n, (unsigned)((rmax + kWoodRows - 1) / kWoodRows)), 256, 0, st>>>(M.subs, a);
  k_wood_s64<<<a.n, 256, 0, st>>>(a);
  k_wood_y64<<<dim3((unsigned)a.n, (unsigned)((a.max_n + 63) / 64)), 256, 0, st>>>(M, a, dst);
  if (!cbuf) return 4;
  k_wood_cb64<<<dim3((unsigned)a.n, (unsigned)((a.max_copy + 255) / 256)), 256, 0, st>>>(M, a, cbuf);
  return 5;
}

}  // namespace tfeti
